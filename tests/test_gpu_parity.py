"""CUDA path against the FP64 oracle, element by element, through the C ABI.

Tolerances (relative L2 per column or field unless stated):
* assembly and right-hand sides: bit-exact (same float64 operations, no
  contraction);
* float64 operator action: 1e-13 (different summation order only);
* float32 operator action on random fields: 2e-6 (a few float32 roundings of
  terms whose magnitude is that of the result);
* float64 combination: 1e-14; bfloat16x3 combination: 1e-6 (three 8-bit
  planes carry 24 bits of the basis; float32 accumulation);
* basis U: 1e-10 for the FP64 path at rtol 1e-12 (kappa ~ 7e3 times the
  residual), 1e-9 for the mixed path refined to rtol 1e-12;
* generated pairs: e_T, e_pair <= 1e-10 (FP64 path), <= 1e-6 (mixed path,
  fields stored in float32).
"""
import numpy as np
import pytest
import torch

from oracle import blockoa_oracle as orc
from paper_2510_23221_gb300 import blockoa as bo
from paper_2510_23221_gb300 import pipeline as pl
from paper_2510_23221_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_23221_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def relcols(a, b, axis=0):
    nb = np.linalg.norm(b, axis=axis)
    return np.linalg.norm(a - b, axis=axis) / np.where(nb > 0, nb, 1.0)


def small_chips():
    return [
        synth.random_small_chip(101, 3, 5, 2),
        synth.random_small_chip(102, 33, 17, 5, h_top=3e4, h_bottom=2e3),
        synth.random_small_chip(103, 9, 4, 3, h_top=0.0, h_side=5e3),
        synth.random_small_chip(104, 7, 6, 3, h_top=1e4, h_bottom=1e3, h_side=1e3, layer_nz=[2, 1, 3]),
        synth.reference_stack_chip(),
        # faces held at the reference temperature (h = inf): all faces, and
        # Robin top and bottom (h = 3e4) with held sides
        synth.random_small_chip(107, 11, 7, 4, h_top=np.inf, h_bottom=np.inf, h_side=np.inf),
        synth.random_small_chip(108, 13, 9, 3, h_top=3e4, h_bottom=3e4, h_side=np.inf),
    ]


# ---------------------------------------------------------------- assembly / rhs
@pytest.mark.parametrize("idx", range(len(small_chips())))
def test_assemble_bitexact(idx):
    chip = small_chips()[idx]
    op = bo.assemble([chip])
    got = bo.export_conductances(op, 0)
    ref = orc.face_conductances(chip)
    for k in ("gx", "gy", "gz", "gb"):
        assert np.array_equal(got[k], ref[k]), k


def test_assemble_batched_uneven_bitexact():
    chips = small_chips()
    op = bo.assemble(chips)
    off = 0
    for c, chip in enumerate(chips):
        assert op.sizes[c]["off"] == off and op.sizes[c]["n"] == chip.n
        off += chip.n
        got = bo.export_conductances(op, c)
        ref = orc.face_conductances(chip)
        for k in ("gx", "gy", "gz", "gb"):
            assert np.array_equal(got[k], ref[k])


def test_build_rhs_exact():
    chips = small_chips()[:3]
    rng = np.random.default_rng(5)
    s = 5
    dens = [np.stack([synth.rect_power_map(rng, c.nx, c.ny) for _ in range(s)]) for c in chips]
    op = bo.assemble(chips)
    B = torch.empty(op.n_total * s, dtype=torch.float64, device="cuda")
    bo.build_rhs(op, cuda(np.concatenate([d.ravel() for d in dens])), B, s)
    Bh = B.cpu().numpy()
    for c, chip in enumerate(chips):
        sz = op.sizes[c]
        assert np.array_equal(Bh[sz["off"] * s:(sz["off"] + sz["n"]) * s].reshape(-1, s),
                              orc.rhs(chip, dens[c]))


# ---------------------------------------------------------------- operator action
@pytest.mark.parametrize("idx", range(len(small_chips())))
def test_apply_fp64(idx):
    chip = small_chips()[idx]
    M = 7
    T = np.random.default_rng(idx).standard_normal((M, chip.n))
    op = bo.assemble([chip])
    q = torch.empty(M * chip.n, dtype=torch.float64, device="cuda")
    bo.apply_operator(op, cuda(T.ravel()), q, M, bo.FP64)
    ref = orc.apply_operator(orc.assemble(chip), T)
    assert np.all(relcols(q.cpu().numpy().reshape(M, -1), ref, axis=1) < 1e-13)


@pytest.mark.parametrize("idx", range(len(small_chips())))
def test_apply_fp32(idx):
    chip = small_chips()[idx]
    M = 9
    T = np.random.default_rng(idx).standard_normal((M, chip.n)).astype(np.float32)
    op = bo.assemble([chip])
    q = torch.empty(M * chip.n, dtype=torch.float32, device="cuda")
    bo.apply_operator(op, cuda(T.ravel()), q, M, bo.MIXED)
    ref = orc.apply_operator(orc.assemble(chip), T.astype(np.float64))
    assert np.all(relcols(q.cpu().numpy().astype(np.float64).reshape(M, -1), ref, axis=1) < 2e-6)


@pytest.mark.parametrize("precision", [bo.FP64, bo.MIXED])
@pytest.mark.parametrize("nx,ny", [(37, 21), (36, 20), (260, 9)])
def test_layered_and_per_cell_forms_agree_bitwise(precision, nx, ny):
    """A layered chip and the same chip given cell by cell give the same q
    (aligned layered chips take the vectorised kernel, the rest the scalar one)."""
    layered = synth.random_small_chip(201, nx, ny, 4, h_top=2e4, h_side=3e3)
    per_cell = synth.random_small_chip(201, nx, ny, 4, h_top=2e4, h_side=3e3)
    per_cell.k_cell = layered.cell_k()
    M = 11
    dt = torch.float64 if precision == bo.FP64 else torch.float32
    T = torch.randn(M * layered.n, dtype=dt, device="cuda")
    q1 = torch.empty_like(T)
    q2 = torch.empty_like(T)
    bo.apply_operator(bo.assemble([layered]), T, q1, M, precision)
    bo.apply_operator(bo.assemble([per_cell]), T, q2, M, precision)
    assert torch.equal(q1, q2)


def test_apply_nonuniform_per_cell_conductivity():
    chip = synth.random_small_chip(202, 19, 14, 3, h_top=1e4, h_side=2e3)
    rng = np.random.default_rng(202)
    chip.k_cell = np.exp(rng.uniform(0, np.log(400), (chip.nz, chip.ny, chip.nx)))
    op = bo.assemble([chip])
    got = bo.export_conductances(op, 0)
    ref = orc.face_conductances(chip)
    for k in ("gx", "gy", "gz", "gb"):
        assert np.array_equal(got[k], ref[k])
    M = 5
    T = np.random.default_rng(3).standard_normal((M, chip.n))
    q = torch.empty(M * chip.n, dtype=torch.float64, device="cuda")
    bo.apply_operator(op, cuda(T.ravel()), q, M, bo.FP64)
    assert np.all(relcols(q.cpu().numpy().reshape(M, -1), orc.apply_operator(orc.assemble(chip), T), axis=1) < 1e-13)
    B = np.random.default_rng(4).uniform(0, 1e-2, (chip.n, 4))
    (X,), (st,) = _solve([chip], [B], 4, bo.MIXED, 1e-11)
    assert st.status == bo.OK
    assert np.all(relcols(X, np.linalg.solve(orc.assemble(chip).toarray(), B)) < 1e-8)


def test_apply_batched_fields_layout():
    chips = small_chips()
    M = 3
    op = bo.assemble(chips)
    rng = np.random.default_rng(9)
    Ts = [rng.standard_normal((M, c.n)) for c in chips]
    q = torch.empty(op.n_total * M, dtype=torch.float64, device="cuda")
    bo.apply_operator(op, cuda(np.concatenate([t.ravel() for t in Ts])), q, M, bo.FP64)
    qh = q.cpu().numpy()
    for c, chip in enumerate(chips):
        sz = op.sizes[c]
        got = qh[sz["off"] * M:(sz["off"] + sz["n"]) * M].reshape(M, -1)
        assert np.all(relcols(got, orc.apply_operator(orc.assemble(chip), Ts[c]), axis=1) < 1e-13)


# ---------------------------------------------------------------- combination
@pytest.mark.parametrize("s,M", [(8, 64), (3, 5), (32, 100), (64, 33), (32, 600), (17, 513)])
def test_combine(s, M):
    chip = synth.random_small_chip(7, 21, 13, 3)
    rng = np.random.default_rng(s * 100 + M)
    U = rng.standard_normal((chip.n, s)) * 10.0 ** rng.uniform(-3, 3, s)
    C = synth.coefficients(rng, s, M)
    op = bo.assemble([chip])
    ref = orc.combine(U, C)
    T64 = torch.empty(M * chip.n, dtype=torch.float64, device="cuda")
    bo.combine(op, cuda(U.ravel()), cuda(C.ravel()), T64, s, M, bo.FP64)
    assert np.all(relcols(T64.cpu().numpy().reshape(M, -1), ref, axis=1) < 1e-14)
    T32 = torch.empty(M * chip.n, dtype=torch.float32, device="cuda")
    bo.combine(op, cuda(U.ravel()), cuda(C.ravel()), T32, s, M, bo.MIXED)
    assert np.all(relcols(T32.cpu().numpy().astype(np.float64).reshape(M, -1), ref, axis=1) < 1e-6)


@pytest.mark.parametrize("precision", [bo.FP64, bo.MIXED])
def test_q_by_linearity(precision):
    """q = (A U) C -- blockoa_apply_basis then blockoa_combine -- equals the
    oracle's A (U C) to the combination's rounding (1e-13 in float64, 1e-6
    with float32 fields; the identity itself is pinned on the oracle), and
    AU matches the oracle's sparse product to summation order."""
    chip = synth.random_small_chip(7, 21, 13, 3)
    s, M = 8, 40
    rng = np.random.default_rng(5)
    U = rng.standard_normal((chip.n, s)) * 10.0 ** rng.uniform(-3, 3, s)
    C = synth.coefficients(rng, s, M)
    op = bo.assemble([chip])
    A = orc.assemble(chip)
    AU = torch.empty(chip.n * s, dtype=torch.float64, device="cuda")
    bo.apply_basis(op, cuda(U.ravel()), AU, s)
    assert np.all(relcols(AU.cpu().numpy().reshape(-1, s), A @ U) < 1e-13)
    q_ref = orc.apply_operator(A, orc.combine(U, C))
    q = torch.empty(M * chip.n, dtype=torch.float64 if precision == bo.FP64 else torch.float32, device="cuda")
    bo.combine(op, AU, cuda(C.ravel()), q, s, M, precision)
    tol = 1e-13 if precision == bo.FP64 else 1e-6
    assert np.all(relcols(q.cpu().numpy().astype(np.float64).reshape(M, -1), q_ref, axis=1) < tol)


@pytest.mark.parametrize("precision", [bo.FP64, bo.MIXED])
def test_combine_with_noise(precision):
    """The epsilon term of Eq. 5: T = U C + epsilon with epsilon from the
    oracle's own Philox4x64-10 at the global cell index; two chips so that
    the second chip's cells are numbered after the first's.  The noise is
    the same number on both sides, so the tolerances are those of U C."""
    chips = [synth.random_small_chip(7, 21, 13, 3), synth.random_small_chip(8, 9, 11, 2)]
    s, M, seed, amp = 8, 37, 2024, 0.01
    rng = np.random.default_rng(6)
    op = bo.assemble(chips)
    Us = [rng.standard_normal((c.n, s)) for c in chips]
    Cs = [synth.coefficients(rng, s, M) for c in chips]
    T = torch.empty(M * op.n_total, dtype=torch.float64 if precision == bo.FP64 else torch.float32,
                    device="cuda")
    bo.combine(op, cuda(np.concatenate([u.ravel() for u in Us])), cuda(np.concatenate([c.ravel() for c in Cs])),
               T, s, M, precision, noise_seed=seed, noise_amp=amp)
    Th = T.cpu().numpy().astype(np.float64)
    tol = 1e-14 if precision == bo.FP64 else 1e-6
    for c, chip in enumerate(chips):
        off = op.sizes[c]["off"]
        ref = orc.combine(Us[c], Cs[c]) + orc.noise(seed, np.arange(off, off + chip.n), M, amp)
        got = Th[off * M:(off + chip.n) * M].reshape(M, chip.n)
        assert np.all(relcols(got, ref, axis=1) < tol)
    with pytest.raises(bo.BlockoaError):
        bo.combine(op, cuda(np.concatenate([u.ravel() for u in Us])), cuda(np.concatenate([c.ravel() for c in Cs])),
                   T, s, M, precision, noise_seed=seed, noise_amp=-1.0)


@pytest.mark.parametrize("precision", [bo.FP64, bo.MIXED])
def test_gaussian_noise_matches_oracle(precision):
    """The Gaussian epsilon (Sec. V-D's noise study) against the oracle's
    noise_gaussian: with a zero basis the fields are the noise itself, so the
    two are compared element by element (float64: a few roundings of
    sigma-sized numbers; float32: evaluated in float32 from u1, u2 rounded
    once, |eps| <= 8.6 sigma, so within 1e-5 sigma); with a random basis the
    noisy field against U C + epsilon at the combination's own tolerance."""
    chips = [synth.random_small_chip(17, 19, 11, 3), synth.random_small_chip(18, 7, 13, 2)]
    s, M, seed, sigma = 8, 41, 4242, 0.05
    rng = np.random.default_rng(16)
    op = bo.assemble(chips)
    fdt = torch.float64 if precision == bo.FP64 else torch.float32
    Cs = [synth.coefficients(rng, s, M) for _ in chips]
    Cd = cuda(np.concatenate([c.ravel() for c in Cs]))
    T = torch.empty(M * op.n_total, dtype=fdt, device="cuda")
    bo.combine(op, torch.zeros(op.n_total * s, dtype=torch.float64, device="cuda"), Cd, T, s, M, precision,
               noise_seed=seed, noise_amp=sigma, noise_kind=bo.NOISE_GAUSSIAN)
    Th = T.cpu().numpy().astype(np.float64)
    atol = 1e-13 * sigma if precision == bo.FP64 else 1e-5 * sigma
    for c, chip in enumerate(chips):
        off = op.sizes[c]["off"]
        ref = orc.noise_gaussian(seed, np.arange(off, off + chip.n), M, sigma)
        got = Th[off * M:(off + chip.n) * M].reshape(M, chip.n)
        assert np.max(np.abs(got - ref)) <= atol, np.max(np.abs(got - ref))
    Us = [rng.standard_normal((c.n, s)) for c in chips]
    bo.combine(op, cuda(np.concatenate([u.ravel() for u in Us])), Cd, T, s, M, precision,
               noise_seed=seed, noise_amp=sigma, noise_kind=bo.NOISE_GAUSSIAN)
    Th = T.cpu().numpy().astype(np.float64)
    tol = 1e-14 if precision == bo.FP64 else 1e-6
    for c, chip in enumerate(chips):
        off = op.sizes[c]["off"]
        ref = orc.combine(Us[c], Cs[c]) + orc.noise_gaussian(seed, np.arange(off, off + chip.n), M, sigma)
        got = Th[off * M:(off + chip.n) * M].reshape(M, chip.n)
        assert np.all(relcols(got, ref, axis=1) < tol)


@pytest.mark.parametrize("precision", [bo.FP64, bo.MIXED])
def test_normalised_weights_match_oracle(precision):
    """Eq. 5's normalised weights alpha_im = C_im / sum_j C_jm against the
    oracle's combine_normalized (with and without uniform noise added
    afterwards), and the guard on weights that sum to ~0."""
    chips = [synth.random_small_chip(27, 23, 9, 3), synth.random_small_chip(28, 8, 8, 4)]
    s, M = 12, 300
    rng = np.random.default_rng(26)
    op = bo.assemble(chips)
    fdt = torch.float64 if precision == bo.FP64 else torch.float32
    Us = [rng.standard_normal((c.n, s)) for c in chips]
    Cs = [synth.coefficients(rng, s, M) + 0.0 for _ in chips]
    Ud = cuda(np.concatenate([u.ravel() for u in Us]))
    Cd = cuda(np.concatenate([c.ravel() for c in Cs]))
    T = torch.empty(M * op.n_total, dtype=fdt, device="cuda")
    tol = 1e-13 if precision == bo.FP64 else 2e-6
    for amp in (0.0, 0.01):
        bo.combine(op, Ud, Cd, T, s, M, precision, normalize=True, noise_seed=9, noise_amp=amp)
        Th = T.cpu().numpy().astype(np.float64)
        for c, chip in enumerate(chips):
            off = op.sizes[c]["off"]
            ref = orc.combine_normalized(Us[c], Cs[c])
            if amp:
                ref = ref + orc.noise(9, np.arange(off, off + chip.n), M, amp)
            got = Th[off * M:(off + chip.n) * M].reshape(M, chip.n)
            assert np.all(relcols(got, ref, axis=1) < tol), relcols(got, ref, axis=1).max()
    # a field whose weights cancel exactly is refused
    Cbad = [c.copy() for c in Cs]
    Cbad[1][:, 7] = 0.0
    Cbad[1][0, 7], Cbad[1][1, 7] = 1.5, -1.5
    with pytest.raises(bo.BlockoaError) as ei:
        bo.combine(op, Ud, cuda(np.concatenate([c.ravel() for c in Cbad])), T, s, M, precision, normalize=True)
    assert ei.value.code == bo.ERR_INVALID


def test_residual_ratio_matches_oracle():
    """The warm start's fallback test, ||B_j - A X_j|| / ||B_j|| per chip and
    column, against the oracle's operator; a zero column of B reads 0 when
    X is zero there and +inf otherwise."""
    chips = [synth.random_small_chip(37, 19, 13, 4), synth.random_small_chip(38, 9, 30, 2, h_side=2e3)]
    s = 11
    rng = np.random.default_rng(36)
    op = bo.assemble(chips)
    Bs = [rng.standard_normal((c.n, s)) for c in chips]
    Xs = [rng.standard_normal((c.n, s)) for c in chips]
    Bs[1][:, 4] = 0.0
    Xs[1][:, 4] = 0.0
    Bs[0][:, 7] = 0.0
    r = torch.empty(op.n_chips * s, dtype=torch.float64, device="cuda")
    bo.residual_ratio(op, cuda(np.concatenate([b.ravel() for b in Bs])),
                      cuda(np.concatenate([x.ravel() for x in Xs])), s, r)
    got = r.cpu().numpy().reshape(op.n_chips, s)
    for c, chip in enumerate(chips):
        A = orc.assemble(chip)
        num = np.linalg.norm(Bs[c] - A @ Xs[c], axis=0)
        den = np.linalg.norm(Bs[c], axis=0)
        for j in range(s):
            if den[j] > 0:
                assert abs(got[c, j] - num[j] / den[j]) <= 1e-12 * num[j] / den[j]
            else:
                assert got[c, j] == (0.0 if num[j] == 0 else np.inf)


def test_fno_basis_scales_and_transposes():
    from paper_2510_23221_gb300 import fno
    chips = [synth.random_small_chip(47, 6, 5, 3), synth.random_small_chip(48, 4, 7, 2)]
    s = 5
    rng = np.random.default_rng(46)
    op = bo.assemble(chips)
    y = rng.standard_normal(op.n_total * s).astype(np.float32)
    scale = rng.uniform(0.5, 2.0, op.n_chips * s)
    X = torch.empty(op.n_total * s, dtype=torch.float64, device="cuda")
    fno.basis(op, cuda(y), cuda(scale), s, X)
    got = X.cpu().numpy()
    for c in range(op.n_chips):
        off, n = op.sizes[c]["off"], op.sizes[c]["n"]
        yc = y[off * s:(off + n) * s].reshape(s, n).astype(np.float64)
        ref = (yc * scale[c * s:(c + 1) * s, None]).T
        assert np.array_equal(got[off * s:(off + n) * s].reshape(n, s), ref)


@pytest.mark.parametrize("case", ["mixed_small", "chip128_ragged_M", "wide_rows_fallback"])
def test_fused_combine_apply_matches_the_two_calls(case):
    """blockoa_combine_apply: T bitwise equal to blockoa_combine's, q within
    float32 rounding of blockoa_apply_operator on that T, and against the
    oracle: e_T to U C and e_pair with the oracle's operator."""
    if case == "mixed_small":
        chips = [synth.random_small_chip(57, 37, 21, 3), synth.reference_stack_chip(),
                 synth.random_small_chip(58, 5, 9, 4, h_top=3e4, h_bottom=2e3, h_side=5e2)]
        s, M = 17, 131
    elif case == "chip128_ragged_M":
        chips = [synth.random_small_chip(59, 128, 16, 4)]
        s, M = 32, 65
    else:
        chips = [synth.random_small_chip(60, 150, 6, 2), synth.random_small_chip(61, 9, 7, 3)]
        s, M = 8, 70
    rng = np.random.default_rng(56)
    op = bo.assemble(chips)
    Us = [rng.standard_normal((c.n, s)) for c in chips]
    Cs = [synth.coefficients(rng, s, M) for _ in chips]
    Ud = cuda(np.concatenate([u.ravel() for u in Us]))
    Cd = cuda(np.concatenate([c.ravel() for c in Cs]))
    T1 = torch.empty(M * op.n_total, dtype=torch.float32, device="cuda")
    q1 = torch.empty_like(T1)
    bo.combine(op, Ud, Cd, T1, s, M, bo.MIXED)
    bo.apply_operator(op, T1, q1, M, bo.MIXED)
    T2 = torch.full_like(T1, float("nan"))
    q2 = torch.full_like(T1, float("nan"))
    bo.combine_apply(op, Ud, Cd, T2, q2, s, M)
    assert torch.equal(T1, T2)
    q1h, q2h = q1.cpu().numpy().astype(np.float64), q2.cpu().numpy().astype(np.float64)
    T2h = T2.cpu().numpy().astype(np.float64)
    for c, chip in enumerate(chips):
        off, n = op.sizes[c]["off"], op.sizes[c]["n"]
        a = q1h[off * M:(off + n) * M].reshape(M, n)
        b = q2h[off * M:(off + n) * M].reshape(M, n)
        assert np.all(relcols(b, a, axis=1) < 2e-6)
        A = orc.assemble(chip)
        Tc = T2h[off * M:(off + n) * M].reshape(M, n)
        e = orc.pair_errors(A, Us[c], Cs[c], Tc, b)
        assert e["e_T"].max() <= 1e-6 and e["e_pair"].max() <= 1e-6, (e["e_T"].max(), e["e_pair"].max())


def test_apply_basis_rejects_bad_arguments():
    op = bo.assemble([synth.random_small_chip(8, 5, 4, 2)])
    with pytest.raises(bo.BlockoaError):
        bo.apply_basis(op, torch.zeros(20 * 4, dtype=torch.float64, device="cuda"),
                       torch.zeros(20 * 4, dtype=torch.float64, device="cuda"), 0)


# ---------------------------------------------------------------- block solve
def _solve(chips, B_list, s, precision, rtol, **kw):
    op = bo.assemble(chips)
    B = cuda(np.concatenate([b.ravel() for b in B_list]))
    X = torch.empty_like(B)
    stats = bo.block_solve(op, B, X, s, rtol=rtol, precision=precision, **kw)
    Xh = X.cpu().numpy()
    out = []
    for c in range(len(chips)):
        sz = op.sizes[c]
        out.append(Xh[sz["off"] * s:(sz["off"] + sz["n"]) * s].reshape(-1, s))
    return out, stats


@pytest.mark.parametrize("precision", [bo.FP64, bo.MIXED])
@pytest.mark.parametrize("idx", [0, 1, 2, 3, 5, 6])
def test_block_solve_tiny_vs_dense(idx, precision):
    chip = small_chips()[idx]
    B = np.random.default_rng(idx).uniform(0, 1e-2, (chip.n, 3))
    # float64's attainable true residual on these grids is ~1e-12 (kappa ~ 1e4)
    (X,), (st,) = _solve([chip], [B], 3, precision, 1e-11)
    assert st.status == bo.OK and st.relres_max <= 1e-11
    ref = np.linalg.solve(orc.assemble(chip).toarray(), B)
    assert np.all(relcols(X, ref) < 1e-9)


@pytest.mark.parametrize("precision", [bo.FP64, bo.MIXED])
def test_block_solve_reference_stack(precision):
    w = synth.small_fp64_workload()
    chip = w.chips[0]
    A = orc.assemble(chip)
    B = orc.rhs(chip, w.density[0])
    U_or, info = orc.block_cg(A, B, rtol=1e-12)
    (X,), (st,) = _solve([chip], [B], 8, precision, 1e-12)
    assert st.status == bo.OK and st.relres_max <= 1e-12
    # the oracle's CSR residual and the kernel's difference-form residual
    # each carry ~1e-13 of float64 rounding at this attainable-accuracy level
    true_rel = relcols(A @ X, B)
    assert np.all(true_rel <= 1.5e-12)
    assert np.all(relcols(X, U_or) < (1e-10 if precision == bo.FP64 else 1e-9))
    if precision == bo.FP64:
        assert abs(st.iters - info["iters"]) <= 8, (st.iters, info["iters"])


def test_block_solve_ragged_tiles_several_units():
    """48x40x6 grid (ragged against every tile shape), s = 12 padded to 16."""
    chip = synth.random_small_chip(55, 48, 40, 6)
    rng = np.random.default_rng(55)
    dens = np.stack([synth.power_maps(rng, 48, 40, 1, True)[0] for _ in range(12)])
    A = orc.assemble(chip)
    B = orc.rhs(chip, dens)
    U_or, _ = orc.block_cg(A, B, rtol=1e-12)
    for precision in (bo.FP64, bo.MIXED):
        (X,), (st,) = _solve([chip], [B], 12, precision, 1e-12)
        assert st.status == bo.OK
        assert np.all(relcols(A @ X, B) <= 1.5e-12)
        assert np.all(relcols(X, U_or) < 1e-9)


@pytest.mark.parametrize("s", [1, 5, 13, 33, 64])
def test_block_solve_column_counts(s):
    chip = synth.random_small_chip(60 + s, 11, 9, 4)
    B = np.random.default_rng(s).uniform(0, 1e-2, (chip.n, s))
    (X,), (st,) = _solve([chip], [B], s, bo.MIXED, 1e-11)
    assert st.status == bo.OK
    ref = np.linalg.solve(orc.assemble(chip).toarray(), B)
    assert np.all(relcols(X, ref) < 1e-8)


def test_block_solve_batched_uneven():
    chips = small_chips()
    rng = np.random.default_rng(77)
    Bs = [rng.uniform(0, 1e-2, (c.n, 4)) for c in chips]
    for precision in (bo.FP64, bo.MIXED):
        Xs, stats = _solve(chips, Bs, 4, precision, 1e-12)
        for c, chip in enumerate(chips):
            assert stats[c].status == bo.OK
            ref = np.linalg.solve(orc.assemble(chip).toarray(), Bs[c])
            assert np.all(relcols(Xs[c], ref) < 1e-9)


@pytest.mark.parametrize("precision", [bo.FP64, bo.MIXED])
def test_jacobi_preconditioned_solve(precision):
    """Diagonal preconditioning changes the iteration, not the solution."""
    w = synth.small_fp64_workload()
    chip = w.chips[0]
    A = orc.assemble(chip)
    B = orc.rhs(chip, w.density[0])
    U_or, info = orc.block_cg(A, B, rtol=1e-12)
    (X,), (st,) = _solve([chip], [B], 8, precision, 1e-12, precond=bo.PRECOND_JACOBI)
    assert st.status == bo.OK and st.relres_max <= 1e-12
    assert np.all(relcols(X, U_or) < 1e-9)
    chips = small_chips()
    rng = np.random.default_rng(78)
    Bs = [rng.uniform(0, 1e-2, (c.n, 4)) for c in chips]
    Xs, stats = _solve(chips, Bs, 4, precision, 1e-11, precond=bo.PRECOND_JACOBI)
    for c, chip in enumerate(chips):
        assert stats[c].status == bo.OK
        ref = np.linalg.solve(orc.assemble(chip).toarray(), Bs[c])
        assert np.all(relcols(Xs[c], ref) < 1e-8)


@pytest.mark.parametrize("precond", [bo.PRECOND_NONE, bo.PRECOND_JACOBI])
def test_mixed_with_fp64_cholesky_small_solves(precond):
    """The mixed loop with float64 Cholesky small solves reaches the same basis."""
    w = synth.small_fp64_workload()
    chip = w.chips[0]
    A = orc.assemble(chip)
    B = orc.rhs(chip, w.density[0])
    U_or, _ = orc.block_cg(A, B, rtol=1e-12)
    (X,), (st,) = _solve([chip], [B], 8, bo.MIXED, 1e-12, precond=precond,
                         small_solve=bo.SMALL_FP64_CHOLESKY)
    assert st.status == bo.OK and st.relres_max <= 1e-12
    assert np.all(relcols(X, U_or) < 1e-9)
    chips = small_chips()
    rng = np.random.default_rng(79)
    Bs = [rng.uniform(0, 1e-2, (c.n, 12)) for c in chips]
    Xs, stats = _solve(chips, Bs, 12, bo.MIXED, 1e-11, precond=precond, small_solve=bo.SMALL_FP64_CHOLESKY)
    for c, chip in enumerate(chips):
        assert stats[c].status == bo.OK
        ref = np.linalg.solve(orc.assemble(chip).toarray(), Bs[c])
        assert np.all(relcols(Xs[c], ref) < 1e-8)


@pytest.mark.parametrize("pc", [bo.PRECOND_ZLINE, bo.PRECOND_ZLINE2])
@pytest.mark.parametrize("precision", [bo.FP64, bo.MIXED])
def test_zline_preconditioned_solve(precision, pc):
    """z-line preconditioning (one or two steps) changes the iteration, not
    the solution: the reference stack at 1e-12 against the oracle, and uneven
    chips (several layer counts, multi-cell layers, ragged column tiles)
    against dense solves."""
    w = synth.small_fp64_workload()
    chip = w.chips[0]
    A = orc.assemble(chip)
    B = orc.rhs(chip, w.density[0])
    U_or, _ = orc.block_cg(A, B, rtol=1e-12)
    (X,), (st,) = _solve([chip], [B], 8, precision, 1e-12, precond=pc)
    assert st.status == bo.OK and st.relres_max <= 1e-12
    assert np.all(relcols(X, U_or) < 1e-9)
    chips = small_chips() + [synth.random_small_chip(105, 37, 21, 5)]
    rng = np.random.default_rng(80)
    for s in (4, 12):
        Bs = [rng.uniform(0, 1e-2, (c.n, s)) for c in chips]
        Xs, stats = _solve(chips, Bs, s, precision, 1e-11, precond=pc)
        for c, ch in enumerate(chips):
            assert stats[c].status == bo.OK, (s, c, stats[c])
            ref = np.linalg.solve(orc.assemble(ch).toarray(), Bs[c])
            assert np.all(relcols(Xs[c], ref) < 1e-8)


@pytest.mark.parametrize("precision", [bo.FP64, bo.MIXED])
def test_two_step_zline_needs_fewer_iterations(precision):
    """The second z-line step (directions from M^-1 (2R - A M^-1 R)) cuts
    the block iterations on a layered chip against one step."""
    chip = synth.single_chip_workload(48, 40, 8, s=8, M=4).chips[0]
    rng = np.random.default_rng(12)
    B = orc.rhs(chip, np.stack([synth.rect_power_map(rng, chip.nx, chip.ny) for _ in range(8)]))
    (X1,), (s1,) = _solve([chip], [B], 8, precision, 1e-9, precond=bo.PRECOND_ZLINE)
    (X2,), (s2,) = _solve([chip], [B], 8, precision, 1e-9, precond=bo.PRECOND_ZLINE2)
    assert s1.status == bo.OK and s2.status == bo.OK
    assert s2.iters < 0.8 * s1.iters, (s1.iters, s2.iters)
    assert np.all(relcols(X2, X1) < 1e-7)


def test_autotune_and_hand_set_unit_sizes_keep_the_results():
    """Unit sizes only regroup the work: after blockoa_autotune, and with
    odd sizes set by hand, solves of an uneven batch still match dense
    solves; the tuning is kept in the operator."""
    chips = [synth.random_small_chip(110 + c, 24 + 7 * c, 18 + 3 * c, 3 + c) for c in range(3)]
    s = 8
    op = bo.assemble(chips)
    t = bo.autotune(op, s, bo.MIXED, bo.PRECOND_ZLINE2)
    assert t["tiles_per_unit"] in (1, 2, 4, 8, 16, 32) and t["ztiles_per_unit"] in (0, 1, 2, 4, 8, 16, 32)
    assert t["ms_per_iter"] > 0
    assert bo.get_tuning(op) == {"tiles_per_unit": t["tiles_per_unit"], "ztiles_per_unit": t["ztiles_per_unit"]}
    rng = np.random.default_rng(21)
    Bs = [rng.uniform(0, 1e-2, (c.n, s)) for c in chips]
    dense = [np.linalg.solve(orc.assemble(c).toarray(), b) for c, b in zip(chips, Bs)]
    for tune in (None, (3, 5)):
        if tune:
            bo.set_tuning(op, *tune)
        B = cuda(np.concatenate([b.ravel() for b in Bs]))
        X = torch.empty_like(B)
        stats = bo.block_solve(op, B, X, s, rtol=1e-11, precision=bo.MIXED, precond=bo.PRECOND_ZLINE2)
        Xh = X.cpu().numpy()
        for c in range(len(chips)):
            assert stats[c].status == bo.OK
            sz = op.sizes[c]
            got = Xh[sz["off"] * s:(sz["off"] + sz["n"]) * s].reshape(-1, s)
            assert np.all(relcols(got, dense[c]) < 1e-8), (tune, c)
    with pytest.raises(bo.BlockoaError):
        bo.set_tuning(op, -1, 0)


def test_reassemble_in_place_matches_fresh_assembly():
    """Re-discretising an operator in place equals a fresh assembly bit for
    bit; a solve on it, reusing the workspace and graph built by a solve on
    the previous chip, matches a dense solve of the new chip; a chip of
    another grid is refused and leaves the operator unchanged."""
    a = synth.random_small_chip(301, 33, 17, 5, h_top=3e4, h_bottom=2e3)
    b = synth.random_small_chip(302, 33, 17, 5, h_top=1e4, h_side=4e3)   # same grid, other k, dz, films
    s = 8
    rng = np.random.default_rng(9)
    op = bo.assemble([a])
    Ba = cuda(rng.uniform(0, 1e-2, (a.n, s)).ravel())
    bo.block_solve(op, Ba, torch.empty_like(Ba), s, rtol=1e-10, precision=bo.MIXED, precond=bo.PRECOND_ZLINE)
    bo.reassemble(op, [b])
    ref = bo.export_conductances(bo.assemble([b]), 0)
    got = bo.export_conductances(op, 0)
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k
    Bb = rng.uniform(0, 1e-2, (b.n, s))
    X = torch.empty(b.n * s, dtype=torch.float64, device="cuda")
    (st,) = bo.block_solve(op, cuda(Bb.ravel()), X, s, rtol=1e-11, precision=bo.MIXED,
                           precond=bo.PRECOND_ZLINE)
    assert st.status == bo.OK
    dense = np.linalg.solve(orc.assemble(b).toarray(), Bb)
    assert np.all(relcols(X.cpu().numpy().reshape(-1, s), dense) < 1e-8)
    with pytest.raises(bo.BlockoaError) as e:
        bo.reassemble(op, [synth.random_small_chip(303, 33, 16, 5)])
    assert e.value.code == bo.ERR_INVALID
    got = bo.export_conductances(op, 0)
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k


@pytest.mark.parametrize("precision", [bo.FP64, bo.MIXED])
def test_independent_columns_are_single_rhs_cg(precision):
    """independent=True runs the s columns as s separate CG solves (the
    per-sample baseline): the solution matches a dense solve; in float64 the
    chip's iteration count is the largest single-column CG count of the
    oracle (within 3), and the block solve of the same columns needs fewer
    iterations (block Krylov shares one space across the columns)."""
    chip = synth.random_small_chip(109, 17, 13, 4)
    s = 6
    rng = np.random.default_rng(11)
    B = np.stack([synth.rect_power_map(rng, chip.nx, chip.ny) for _ in range(s)])
    Bc = orc.rhs(chip, B)
    (X,), (st,) = _solve([chip], [Bc], s, precision, 1e-10, independent=True)
    assert st.status == bo.OK and st.relres_max <= 1e-10
    A = orc.assemble(chip)
    dense = np.linalg.solve(A.toarray(), Bc)
    assert np.all(relcols(X, dense) < 1e-7)
    if precision == bo.FP64:
        single = [orc.block_cg(A, Bc[:, j:j + 1], rtol=1e-10)[1]["iters"] for j in range(s)]
        assert abs(st.iters - max(single)) <= 3, (st.iters, single)
        (_,), (stb,) = _solve([chip], [Bc], s, precision, 1e-10)
        assert stb.iters < st.iters, (stb.iters, st.iters)


@pytest.mark.parametrize("precision,pc", [(bo.MIXED, bo.PRECOND_ZLINE2), (bo.MIXED, bo.PRECOND_JACOBI),
                                          (bo.MIXED, bo.PRECOND_ZLINE), (bo.FP64, bo.PRECOND_NONE),
                                          (bo.FP64, bo.PRECOND_ZLINE2)])
def test_deterministic_solves_repeat_bitwise(precision, pc):
    """deterministic=True: static unit schedules and every partial sum
    reduced in a fixed order -- two solves of the same inputs give the same
    bits and the same iteration counts, on a batch of uneven chips with
    several units each, and reach the dense solution."""
    chips = small_chips()[1:] + [synth.random_small_chip(112, 48, 40, 6), synth.random_small_chip(113, 37, 21, 5)]
    rng = np.random.default_rng(83)
    for s in (5, 12, 32):
        Bs = [rng.uniform(0, 1e-2, (c.n, s)) for c in chips]
        runs = []
        for _ in range(2):
            Xs, stats = _solve(chips, Bs, s, precision, 1e-11, precond=pc, deterministic=True)
            runs.append((Xs, [(st.status, st.iters, st.refine_steps) for st in stats]))
        assert runs[0][1] == runs[1][1], (s, runs[0][1], runs[1][1])
        for a, b in zip(runs[0][0], runs[1][0]):
            assert np.array_equal(a, b)
        for c, ch in enumerate(chips):
            assert runs[0][1][c][0] == bo.OK
            ref = np.linalg.solve(orc.assemble(ch).toarray(), Bs[c])
            assert np.all(relcols(runs[0][0][c], ref) < 1e-8), (s, c)


def test_deterministic_independent_columns():
    """Independent columns (only the Grams' diagonals) in the deterministic
    mode: bitwise repetition and the dense solution."""
    chip = synth.random_small_chip(114, 23, 17, 4)
    s = 20
    rng = np.random.default_rng(14)
    B = np.stack([synth.rect_power_map(rng, chip.nx, chip.ny) for _ in range(s)])
    Bc = orc.rhs(chip, B)
    dense = np.linalg.solve(orc.assemble(chip).toarray(), Bc)
    for precision in (bo.MIXED, bo.FP64):
        runs = [_solve([chip], [Bc], s, precision, 1e-10, independent=True, deterministic=True) for _ in range(2)]
        (X0,), (s0,) = runs[0]
        (X1,), (s1,) = runs[1]
        assert s0.status == bo.OK and (s0.iters, s0.refine_steps) == (s1.iters, s1.refine_steps)
        assert np.array_equal(X0, X1)
        assert np.all(relcols(X0, dense) < 1e-7)


def test_deterministic_headline_chip_repeats_bitwise():
    """The 128 x 128 x 8 chip at s = 32 in the chosen form, deterministic:
    three solves, identical bits and iteration counts."""
    w = synth.single_chip_workload(128, 128, 8, s=32, M=4)
    op = bo.assemble(w.chips)
    B = torch.empty(op.n_total * 32, dtype=torch.float64, device="cuda")
    bo.build_rhs(op, pl.upload(w).density, B, 32)
    outs = []
    for _ in range(3):
        U = torch.empty_like(B)
        st = bo.block_solve(op, B, U, 32, rtol=1e-6, **dict(pl.CHOSEN_SOLVE, deterministic=True))
        assert st[0].status == bo.OK and st[0].relres_max <= 1e-6
        outs.append((U.cpu().numpy(), st[0].iters, st[0].refine_steps))
    for U, it, rf in outs[1:]:
        assert it == outs[0][1] and rf == outs[0][2]
        assert np.array_equal(U, outs[0][0])


def test_deterministic_flag_is_validated():
    op = bo.assemble([synth.random_small_chip(8, 5, 4, 2)])
    B = torch.ones(op.n_total * 4, dtype=torch.float64, device="cuda")
    X = torch.empty_like(B)
    with pytest.raises(bo.BlockoaError):
        bo.block_solve(op, B, X, 4, precision=bo.MIXED, deterministic=2)


def test_zline_needs_columns_that_fit_a_tile():
    chip = synth.random_small_chip(106, 3, 3, 70)          # 70 cells in z > the 64-cell tile at s = 64
    op = bo.assemble([chip])
    B = cuda(np.random.default_rng(1).uniform(0, 1, chip.n * 64))
    with pytest.raises(bo.BlockoaError) as e:
        bo.block_solve(op, B, torch.empty_like(B), 64, precision=bo.MIXED, precond=bo.PRECOND_ZLINE)
    assert e.value.code == bo.ERR_INVALID


def test_deflation_duplicate_and_zero_columns():
    chip = synth.random_small_chip(81, 12, 10, 3)
    B = np.random.default_rng(81).uniform(0, 1e-2, (chip.n, 6))
    B[:, 4] = B[:, 1]
    B[:, 5] = 0.0
    for precision in (bo.FP64, bo.MIXED):
        (X,), (st,) = _solve([chip], [B], 6, precision, 1e-12)
        assert st.status == bo.OK and st.deflated_cols > 0
        assert np.all(X[:, 5] == 0.0)
        assert np.linalg.norm(X[:, 4] - X[:, 1]) <= 1e-10 * np.linalg.norm(X[:, 1])
        ref = np.linalg.solve(orc.assemble(chip).toarray(), B[:, :4])
        assert np.all(relcols(X[:, :4], ref) < 1e-9)


def test_statuses_not_converged_and_breakdown():
    chips = [synth.random_small_chip(91, 10, 10, 3), synth.random_small_chip(92, 8, 9, 4)]
    rng = np.random.default_rng(91)
    Bs = [rng.uniform(0, 1e-2, (c.n, 4)) for c in chips]
    _, stats = _solve(chips, Bs, 4, bo.FP64, 1e-14, maxiter=3, raise_on_error=False)
    assert all(s.status == bo.ERR_NOT_CONVERGED for s in stats)
    assert all(s.iters == 3 for s in stats)
    Bs[1][3, 2] = np.nan
    Xs, stats = _solve(chips, Bs, 4, bo.MIXED, 1e-10, raise_on_error=False)
    assert stats[0].status == bo.OK
    assert stats[1].status == bo.ERR_BREAKDOWN
    ref = np.linalg.solve(orc.assemble(chips[0]).toarray(), Bs[0])
    assert np.all(relcols(Xs[0], ref) < 1e-8)


@pytest.mark.parametrize("precision", [bo.FP64, bo.MIXED])
def test_timeout_status_of_one_chip_is_reported_and_others_converge(precision):
    """A chip whose device state reads ERR_TIMEOUT between polls (what the
    P update's bounded wait leaves when it gives up; injected here from the
    host, nothing on the GPU waits or faults) is reported with that status,
    and the other chips of the operator still converge to the dense
    solution."""
    chips = [small_chips()[i] for i in (1, 2, 3)]
    rng = np.random.default_rng(71)
    Bs = [rng.uniform(0, 1e-2, (c.n, 4)) for c in chips]
    op = bo.assemble(chips)
    B = cuda(np.concatenate([b.ravel() for b in Bs]))
    X = torch.empty_like(B)
    bo.inject_chip_status(op, 1, bo.ERR_TIMEOUT, after_polls=1)
    st = bo.block_solve(op, B, X, 4, rtol=1e-10, precision=precision, check_every=2, raise_on_error=False)
    assert st[1].status == bo.ERR_TIMEOUT
    Xh = X.cpu().numpy()
    for c in (0, 2):
        assert st[c].status == bo.OK and st[c].relres_max <= 1e-10, st[c]
        sz = op.sizes[c]
        got = Xh[sz["off"] * 4:(sz["off"] + sz["n"]) * 4].reshape(-1, 4)
        ref = np.linalg.solve(orc.assemble(chips[c]).toarray(), Bs[c])
        assert np.all(relcols(got, ref) < 1e-8)
    with pytest.raises(bo.BlockoaError):
        bo.inject_chip_status(op, 7, bo.ERR_TIMEOUT)
    # armed once: the next solve is clean
    st = bo.block_solve(op, B, X, 4, rtol=1e-10, precision=precision, check_every=2)
    assert all(x.status == bo.OK for x in st)


def test_invalid_calls_return_invalid():
    chip = synth.random_small_chip(3, 4, 4, 2)
    op = bo.assemble([chip])
    B = torch.zeros(chip.n * 65, dtype=torch.float64, device="cuda")
    with pytest.raises(bo.BlockoaError) as e:
        bo.block_solve(op, B, B.clone(), 65)
    assert e.value.code == bo.ERR_INVALID
    with pytest.raises(bo.BlockoaError) as e:
        bo.block_solve(op, B, B.clone(), 4, rtol=0.0)
    assert e.value.code == bo.ERR_INVALID
    with pytest.raises(bo.BlockoaError) as e:
        bo.block_solve(op, B, B.clone(), 4, precond=7)
    assert e.value.code == bo.ERR_INVALID
    with pytest.raises(bo.BlockoaError) as e:
        bo.block_solve(op, B, B.clone(), 4, small_solve=5)
    assert e.value.code == bo.ERR_INVALID
    T = torch.zeros(chip.n, dtype=torch.float64, device="cuda")
    with pytest.raises(bo.BlockoaError):
        bo.apply_operator(op, T, T, 1, bo.FP64)


# ---------------------------------------------------------------- the paper's 3-D IC (Sec. V-A)
def test_build_rhs_volume_exact():
    """Volumetric sources on two chips of different stacks: bit-exact."""
    chips = [synth.paper_3dic_chip(3, nx=13, ny=14, device_cells=2),
             synth.random_small_chip(4, 9, 7, 3, layer_nz=[2, 1, 2])]
    rng = np.random.default_rng(8)
    s = 5
    qvs = [synth.paper_3dic_sources(rng, chips[0], s),
           rng.uniform(0.0, 1e9, (s, chips[1].nz, chips[1].ny, chips[1].nx))]
    op = bo.assemble(chips)
    B = torch.empty(op.n_total * s, dtype=torch.float64, device="cuda")
    bo.build_rhs_volume(op, cuda(np.concatenate([q.ravel() for q in qvs])), B, s)
    Bh = B.cpu().numpy()
    for c, chip in enumerate(chips):
        sz = op.sizes[c]
        assert np.array_equal(Bh[sz["off"] * s:(sz["off"] + sz["n"]) * s].reshape(-1, s),
                              orc.rhs_volume(chip, qvs[c]))


@pytest.mark.parametrize("precision", [bo.FP64, bo.MIXED])
@pytest.mark.parametrize("boundary", synth.PAPER_BOUNDARIES)
def test_paper_3dic_pipeline(boundary, precision):
    """Two floorplans of the six-layer 3-D IC (copper TSV columns, sources in
    the core and both cache layers) batched in one operator, under each of
    the paper's boundary scenarios: sources, basis, T = U C + epsilon (Eq. 5,
    amplitude 0.01 as in the paper's experiments) and q = A T against the
    oracle, and the pairs' own consistency."""
    chips = [synth.paper_3dic_chip(40 + i, nx=24, ny=20, boundary=boundary, device_cells=2) for i in range(2)]
    s, M, seed, amp = 8, 16, 77, 0.01
    rng = np.random.default_rng(41)
    qvs = [synth.paper_3dic_sources(rng, c, s) for c in chips]
    Cs = [synth.coefficients(rng, s, M) for c in chips]
    op = bo.assemble(chips)
    fdt = torch.float64 if precision == bo.FP64 else torch.float32
    B = torch.empty(op.n_total * s, dtype=torch.float64, device="cuda")
    bo.build_rhs_volume(op, cuda(np.concatenate([q.ravel() for q in qvs])), B, s)
    U = torch.empty_like(B)
    pc = bo.PRECOND_ZLINE2 if precision == bo.MIXED else bo.PRECOND_NONE
    stats = bo.block_solve(op, B, U, s, rtol=1e-12, precision=precision, precond=pc)
    assert all(st.status == bo.OK and st.relres_max <= 1e-12 for st in stats)
    T = torch.empty(M * op.n_total, dtype=fdt, device="cuda")
    q = torch.empty_like(T)
    bo.combine(op, U, cuda(np.concatenate([c.ravel() for c in Cs])), T, s, M, precision,
               noise_seed=seed, noise_amp=amp)
    bo.apply_operator(op, T, q, M, precision)
    e_pair = torch.empty(op.n_chips * M, dtype=torch.float64, device="cuda")
    bo.pair_check(op, T, q, M, precision, e_pair)
    Bh, Uh = B.cpu().numpy(), U.cpu().numpy()
    Th, qh = T.cpu().numpy().astype(np.float64), q.cpu().numpy().astype(np.float64)
    tol_u, tol_f, tol_q = (1e-10, 1e-10, 1e-13) if precision == bo.FP64 else (1e-9, 1e-6, 2e-6)
    for c, chip in enumerate(chips):
        off, n = op.sizes[c]["off"], chip.n
        A = orc.assemble(chip)
        B_or = orc.rhs_volume(chip, qvs[c])
        assert np.array_equal(Bh[off * s:(off + n) * s].reshape(n, s), B_or)
        U_or, info = orc.block_cg(A, B_or, rtol=1e-12)
        assert np.all(relcols(Uh[off * s:(off + n) * s].reshape(n, s), U_or) < tol_u)
        T_or = orc.combine(U_or, Cs[c]) + orc.noise(seed, np.arange(off, off + n), M, amp)
        Tc = Th[off * M:(off + n) * M].reshape(M, n)
        assert np.all(relcols(Tc, T_or, axis=1) < tol_f)
        q_or = orc.apply_operator(A, Tc)          # q of the stored fields
        assert np.all(relcols(qh[off * M:(off + n) * M].reshape(M, n), q_or, axis=1) < tol_q)
    assert float(e_pair.max()) <= (1e-10 if precision == bo.FP64 else 1e-6)


def test_short_buffers_are_refused_before_launch():
    """The library sees only pointers: the binding refuses a tensor smaller
    than the call reads or writes, before anything is launched."""
    chips = [synth.paper_3dic_chip(9, nx=10, ny=9, device_cells=1), synth.random_small_chip(9, 7, 5, 3)]
    op = bo.assemble(chips)
    s, M = 5, 3
    n = op.n_total
    B = torch.zeros(n * s, dtype=torch.float64, device="cuda")
    top = sum(c.nx * c.ny for c in chips)
    with pytest.raises(ValueError):
        bo.build_rhs_volume(op, torch.zeros(top * s, dtype=torch.float64, device="cuda"), B, s)
    with pytest.raises(ValueError):
        bo.build_rhs(op, torch.zeros(top * s - 1, dtype=torch.float64, device="cuda"), B, s)
    with pytest.raises(ValueError):
        bo.block_solve(op, B, B[: n * s - 1], s)
    T = torch.zeros(n * M, dtype=torch.float32, device="cuda")
    C = torch.zeros(len(chips) * s * M, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        bo.combine(op, B, C[:-1], T, s, M, bo.MIXED)
    with pytest.raises(ValueError):
        bo.apply_operator(op, T, T[:-1].clone(), M, bo.MIXED)
    with pytest.raises(ValueError):
        bo.pair_check(op, T, T.clone(), M, bo.MIXED, torch.zeros(len(chips) * M - 1, dtype=torch.float64,
                                                                device="cuda"))
    # the right sizes go through
    bo.build_rhs_volume(op, torch.ones(n * s, dtype=torch.float64, device="cuda"), B, s)
    torch.cuda.synchronize()
    assert float(B.min()) > 0


def test_empty_sizes_are_noops():
    chip = synth.random_small_chip(4, 4, 4, 2)
    op = bo.assemble([chip])
    T = torch.zeros(chip.n, dtype=torch.float64, device="cuda")
    bo.apply_operator(op, T, T.clone(), 0, bo.FP64)
    st = bo.block_solve(op, T, T.clone(), 0)
    assert st[0].status == bo.OK


# ---------------------------------------------------------------- whole path
def test_pipeline_reference_stack_fp64():
    w = synth.small_fp64_workload()
    res = pl.run(w, bo.FP64)
    chip = w.chips[0]
    out = orc.generate(chip, w.density[0], w.coeffs[0], rtol=1e-12)
    T = pl.chip_fields(res, 0, "T").cpu().numpy()
    q = pl.chip_fields(res, 0, "q").cpu().numpy()
    e = orc.pair_errors(out["A"], out["U"], w.coeffs[0], T, q)
    assert np.max(e["e_T"]) <= 1e-10 and np.max(e["e_q"]) <= 1e-10 and np.max(e["e_pair"]) <= 1e-10
    # pair check kernel agrees with the oracle's e_pair
    ep = torch.empty(w.M, dtype=torch.float64, device="cuda")
    bo.pair_check(res.op, res.T, res.q, w.M, bo.FP64, ep)
    assert np.allclose(ep.cpu().numpy(), e["e_pair"], rtol=0, atol=1e-13)


def test_pipeline_reference_stack_mixed():
    w = synth.small_fp64_workload()
    res = pl.run(w, bo.MIXED, rtol=1e-12)
    chip = w.chips[0]
    out = orc.generate(chip, w.density[0], w.coeffs[0], rtol=1e-12)
    T = pl.chip_fields(res, 0, "T").cpu().numpy().astype(np.float64)
    q = pl.chip_fields(res, 0, "q").cpu().numpy().astype(np.float64)
    e = orc.pair_errors(out["A"], out["U"], w.coeffs[0], T, q)
    assert np.max(e["e_T"]) <= 1e-6 and np.max(e["e_pair"]) <= 1e-6
    ep = torch.empty(w.M, dtype=torch.float64, device="cuda")
    bo.pair_check(res.op, res.T, res.q, w.M, bo.MIXED, ep)
    assert np.allclose(ep.cpu().numpy(), e["e_pair"], rtol=1e-6, atol=1e-12)


def test_pipeline_full_size_128x128x8_sampled():
    """The benchmark workload (n = 131072, s = 32, M = 5000, mixed, rtol 1e-6):
    the oracle checks the basis residual, sampled fields of T against U C,
    and sampled q against A T, each with its own float64 arithmetic."""
    w = synth.single_chip_workload()
    res = pl.run(w, bo.MIXED)
    chip = w.chips[0]
    A = orc.assemble(chip)
    B = orc.rhs(chip, w.density[0])
    U = pl.chip_block(res, 0, "U").cpu().numpy()
    assert np.all(relcols(A @ U, B) <= 1.0001e-6)
    T = pl.chip_fields(res, 0, "T")
    q = pl.chip_fields(res, 0, "q")
    C = w.coeffs[0]
    for m in (0, 1, 2047, 2500, 4999):
        Tm = T[m].cpu().numpy().astype(np.float64)
        qm = q[m].cpu().numpy().astype(np.float64)
        ref = U @ C[:, m]
        assert np.linalg.norm(Tm - ref) <= 1e-6 * np.linalg.norm(ref)
        Aq = A @ Tm
        assert np.linalg.norm(Aq - qm) <= 1e-6 * np.linalg.norm(qm)
        # energy balance of the generated pair: net source = Robin loss
        loss = orc.boundary_loss(chip, Tm)[0]
        assert abs(qm.sum() - loss) <= 1e-5 * np.abs(qm).sum()
