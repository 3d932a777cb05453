"""FP64 CPU oracle for the BlocKOA hot path.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
the benchmark's CPU-baseline / reference leg may import this module.  The
product path never calls it; it shares no code with the CUDA library (the
only common import is the seeded input generator, which holds no method
arithmetic).

Everything is plain float64 numpy / scipy, written to be checked by eye
against the paper:

* ``assemble``      -- discretised heat operator A of Eq. 1 / Eq. 2 with the
                       Robin condition of Sec. II-A, as a cell-centred
                       finite-volume 7-point stencil in conservative flux form
                       -div(k grad T) (harmonic face conductances).
* ``rhs``           -- right-hand sides b of Eq. 2: cell power in W from a
                       top-layer power density in W/m^2.
* ``rhs_volume``    -- the same from a volumetric source in W/m^3 anywhere
                       in the stack (the device layers of Sec. V-A's 3-D IC).
* ``block_cg``      -- block conjugate gradient on A X = B for all columns of
                       one chip at once (Eq. 4, Sec. III-A), O'Leary form with
                       Jacobi-scaled pivoted-Cholesky deflation of the s x s
                       Gram matrix.
* ``combine``       -- new temperature fields T = U C (Eq. 5 without the
                       normalisation and noise terms; unknowns are excess
                       temperature, so any C keeps the boundary conditions).
* ``combine_normalized`` -- the same with Eq. 5's normalised weights
                       alpha_im = mu_im / sum_j mu_jm (each field's weights
                       sum to one).
* ``noise``         -- the epsilon term of Eq. 5: uniform noise per cell and
                       field from ``philox4x64_10``, a counter-based generator
                       written from its published definition.
* ``noise_gaussian``-- the Gaussian variant of that noise (Box-Muller from a
                       second Philox stream).
* ``apply_operator``-- operator action q = A T (Eq. 6, Sec. III-C).
* ``pair_errors``   -- relative L2 errors of generated pairs.

Unknowns are excess temperature theta = T - T_ambient (K); rows of A are in
W/K.  Cells are numbered a = (z * ny + y) * nx + x with z = 0 the top layer.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.linalg import solve_triangular

STATUS_OK = 0
STATUS_BREAKDOWN = 3
STATUS_NOT_CONVERGED = 4


# --------------------------------------------------------------------------
# Assembly (Eq. 1 in flux form, Robin faces of Sec. II-A)
# --------------------------------------------------------------------------
def _series(area, half_a, k_a, half_b, k_b):
    """Face conductance between two cell centres: area / (d_a/(2k_a) + d_b/(2k_b)).

    ``half_a`` and ``half_b`` are full cell widths d; the half-cell distance
    d/2 from each centre to the shared face is taken inside.
    """
    return area / (half_a / (2.0 * k_a) + half_b / (2.0 * k_b))


def _robin(area, d, k, h):
    """Boundary conductance of a convective face: area / (d/(2k) + 1/h).

    h = inf is a face held at the reference temperature (Dirichlet, theta =
    0 on the face): 1/h = 0 leaves the half-cell conductance 2 k area / d."""
    return area / (d / (2.0 * k) + 1.0 / h)


def face_conductances(chip):
    """Per-face conductances of the chip, W/K.

    Returns a dict with
      gx [nz][ny][nx-1]  between (z,y,x) and (z,y,x+1), face area dy*dz
      gy [nz][ny-1][nx]  between (z,y,x) and (z,y+1,x), face area dx*dz
      gz [nz-1][ny][nx]  between (z,y,x) and (z+1,y,x), face area dx*dy
      gb [nz][ny][nx]    total Robin conductance of the cell's boundary
                         faces, summed in the order top, bottom, x-low,
                         x-high, y-low, y-high.
    """
    k = chip.cell_k()
    dz = chip.cell_dz()[:, None, None]
    dx, dy = float(chip.dx), float(chip.dy)
    nz, ny, nx = k.shape
    gx = _series(dy * dz, dx, k[:, :, :-1], dx, k[:, :, 1:])
    gy = _series(dx * dz, dy, k[:, :-1, :], dy, k[:, 1:, :])
    gz = _series(dx * dy, dz[:-1], k[:-1], dz[1:], k[1:])
    gb = np.zeros_like(k)
    if chip.h_top > 0:
        gb[0] += _robin(dx * dy, dz[0], k[0], chip.h_top)
    if chip.h_bottom > 0:
        gb[nz - 1] += _robin(dx * dy, dz[nz - 1], k[nz - 1], chip.h_bottom)
    if chip.h_side > 0:
        dzb = np.broadcast_to(dz, k.shape)
        gb[:, :, 0] += _robin(dy * dzb[:, :, 0], dx, k[:, :, 0], chip.h_side)
        gb[:, :, nx - 1] += _robin(dy * dzb[:, :, nx - 1], dx, k[:, :, nx - 1], chip.h_side)
        gb[:, 0, :] += _robin(dx * dzb[:, 0, :], dy, k[:, 0, :], chip.h_side)
        gb[:, ny - 1, :] += _robin(dx * dzb[:, ny - 1, :], dy, k[:, ny - 1, :], chip.h_side)
    return {"gx": gx, "gy": gy, "gz": gz, "gb": gb}


def assemble(chip) -> sp.csr_matrix:
    """Sparse A with (A theta)_a = sum_b G_ab (theta_a - theta_b) + Gb_a theta_a.

    Built face by face: every interior face adds +G to both diagonals and -G
    to both off-diagonal entries, so A is exactly symmetric.
    """
    f = face_conductances(chip)
    nz, ny, nx = chip.nz, chip.ny, chip.nx
    idx = np.arange(chip.n).reshape(nz, ny, nx)
    rows, cols, vals = [], [], []

    def add_faces(a, b, g):
        a, b, g = a.ravel(), b.ravel(), g.ravel()
        rows.extend([a, b, a, b])
        cols.extend([a, b, b, a])
        vals.extend([g, g, -g, -g])

    add_faces(idx[:, :, :-1], idx[:, :, 1:], f["gx"])
    add_faces(idx[:, :-1, :], idx[:, 1:, :], f["gy"])
    add_faces(idx[:-1], idx[1:], f["gz"])
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(f["gb"].ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(chip.n, chip.n))
    return A.tocsr()


def rhs(chip, density) -> np.ndarray:
    """B [n][s]: density (W/m^2) x dx*dy deposited in the top cell row z = 0."""
    density = np.asarray(density, np.float64)
    s = density.shape[0]
    B = np.zeros((chip.n, s))
    area = float(chip.dx) * float(chip.dy)
    top = chip.nx * chip.ny
    B[:top, :] = (density.reshape(s, top) * area).T
    return B


def rhs_volume(chip, qv) -> np.ndarray:
    """B [n][s]: volumetric source qv (W/m^3, [s][nz][ny][nx]) times the cell
    volume dx * dy * dz of each cell's layer (the q of Eq. 1 integrated over
    the cell, Eq. 2).  Plain loop over z-rows."""
    qv = np.asarray(qv, np.float64)
    s = qv.shape[0]
    nxny = chip.nx * chip.ny
    dz = chip.cell_dz()
    q = qv.reshape(s, chip.nz, nxny)
    B = np.zeros((chip.n, s))
    for z in range(chip.nz):
        vol = (float(chip.dx) * float(chip.dy)) * float(dz[z])
        B[z * nxny:(z + 1) * nxny, :] = (q[:, z, :] * vol).T
    return B


def boundary_loss(chip, theta) -> np.ndarray:
    """Heat leaving through Robin faces, sum_a Gb_a theta_a, for theta [n][m]."""
    gb = face_conductances(chip)["gb"].ravel()
    return gb @ np.asarray(theta).reshape(chip.n, -1)


# --------------------------------------------------------------------------
# Block CG with deflation (Eq. 4; block Krylov solve of Sec. III-A)
# --------------------------------------------------------------------------
def scaled_pivoted_cholesky(G, tol):
    """Diagonal-pivoted Cholesky of D G D with D = diag(G)^(-1/2).

    Pivots are taken largest remaining scaled diagonal first (lowest index on
    ties); factorisation stops when the largest remaining pivot is <= tol and
    the remaining columns are deflated.  Returns (kept, L, d): ``kept`` lists
    the kept column indices in pivot order, L is lower triangular with
    (D G D)[kept][:, kept] = L L^T, and d holds the scaling diagonal.
    """
    s = G.shape[0]
    diag = np.diag(G).copy()
    usable = np.isfinite(diag) & (diag > 0)
    d = np.zeros(s)
    d[usable] = 1.0 / np.sqrt(diag[usable])
    W = d[:, None] * G * d[None, :]
    remaining = [j for j in range(s) if usable[j]]
    kept, cols = [], []
    while remaining:
        piv = max(remaining, key=lambda j: (W[j, j], -j))
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
    L = np.stack(cols, axis=1)[kept, :]
    return kept, L, d


def _gram_solve(kept, L, d, Y):
    """Solve G[kept][:, kept] Z = Y[kept] through the scaled factor."""
    dk = d[kept]
    z = solve_triangular(L, dk[:, None] * Y[kept], lower=True)
    z = solve_triangular(L.T, z, lower=False)
    return dk[:, None] * z


def block_cg(A, B, X0=None, rtol=1e-12, maxiter=10000, deflate_tol=1e-14,
             record=None):
    """Block CG for A X = B (all s columns share A and one Krylov space).

    Each iteration: Q = A P; Gamma = P^T Q; factor Gamma with deflation;
    alpha = Gamma^-1 (P^T R); X += P alpha; R -= Q alpha;
    beta = -Gamma^-1 (Q^T R); P = R + P beta.  Deflated columns get zero rows
    in alpha and beta.  Stops when ||R_j|| <= rtol ||B_j|| for every column
    (Sec. V, relative residual norm), or at ``maxiter`` iterations.
    Returns (X, info).
    """
    B = np.asarray(B, np.float64)
    n, s = B.shape
    X = np.zeros((n, s)) if X0 is None else np.array(X0, np.float64, copy=True)
    R = B - A @ X
    P = R.copy()
    bnorm = np.linalg.norm(B, axis=0)
    info = {"status": STATUS_OK, "iters": 0, "deflated": 0}
    it = 0
    while True:
        rnorm = np.linalg.norm(R, axis=0)
        if np.all(rnorm <= rtol * bnorm):
            break
        if not np.all(np.isfinite(rnorm)):
            info["status"] = STATUS_BREAKDOWN
            break
        if it >= maxiter:
            info["status"] = STATUS_NOT_CONVERGED
            break
        Q = A @ P
        G = P.T @ Q
        if not np.all(np.isfinite(G)):
            info["status"] = STATUS_BREAKDOWN
            break
        G = 0.5 * (G + G.T)
        kept, L, d = scaled_pivoted_cholesky(G, deflate_tol)
        if not kept:
            info["status"] = STATUS_BREAKDOWN
            break
        info["deflated"] += s - len(kept)
        alpha = np.zeros((s, s))
        alpha[kept] = _gram_solve(kept, L, d, P.T @ R)
        X += P @ alpha
        R -= Q @ alpha
        beta = np.zeros((s, s))
        beta[kept] = -_gram_solve(kept, L, d, Q.T @ R)
        P = R + P @ beta
        it += 1
        if record is not None:
            record.append(X.copy())
    info["iters"] = it
    true_r = B - A @ X
    with np.errstate(invalid="ignore", divide="ignore"):
        rel = np.where(bnorm > 0, np.linalg.norm(true_r, axis=0) / np.where(bnorm > 0, bnorm, 1), 0.0)
    info["relres"] = rel
    return X, info


# --------------------------------------------------------------------------
# Combination (Eq. 5) and operator action (Eq. 6)
# --------------------------------------------------------------------------
def combine(U, C) -> np.ndarray:
    """T [M][n]: field m is sum_i C[i, m] U[:, i]."""
    return (np.asarray(U, np.float64) @ np.asarray(C, np.float64)).T.copy()


def combine_normalized(U, C) -> np.ndarray:
    """T [M][n] with the normalised weights of Eq. 5: for field m the weights
    are alpha_im = C[i, m] / sum_j C[j, m], and field m is
    sum_i alpha_im U[:, i]."""
    C = np.asarray(C, np.float64)
    alpha = C / C.sum(axis=0, keepdims=True)
    return combine(U, alpha)


# ---------------------------------------------------------------- noise (Eq. 5's epsilon)
_PHILOX_M = (0xD2E7470EE14C6C93, 0xCA5A826395121157)
_PHILOX_W = (0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B)
_MASK64 = (1 << 64) - 1


def philox4x64_10(counter, key):
    """One block of the Philox4x64-10 generator (Salmon, Moraes, Dror, Shaw,
    SC 2011), written from its definition with Python integers: ten rounds;
    before every round after the first the key is bumped by the Weyl
    constants; a round maps (c0, c1, c2, c3) to
    (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))."""
    c = [int(x) & _MASK64 for x in counter]
    k0, k1 = (int(x) & _MASK64 for x in key)
    for r in range(10):
        if r > 0:
            k0 = (k0 + _PHILOX_W[0]) & _MASK64
            k1 = (k1 + _PHILOX_W[1]) & _MASK64
        p0 = _PHILOX_M[0] * c[0]
        p1 = _PHILOX_M[1] * c[2]
        c = [(p1 >> 64) ^ c[1] ^ k0, p1 & _MASK64, (p0 >> 64) ^ c[3] ^ k1, p0 & _MASK64]
    return c


def noise(seed, cells, M, amp) -> np.ndarray:
    """epsilon [M][len(cells)] of the combination: for global cell index a and
    field m, word m % 4 of Philox4x64-10 at counter (a, m // 4, 0, 0) and key
    (seed, 0) gives u = (w >> 11) 2^-53 in [0, 1) and epsilon = amp (2u - 1).
    Plain loops: small cases only."""
    out = np.empty((M, len(cells)))
    for i, a in enumerate(cells):
        for g in range((M + 3) // 4):
            w = philox4x64_10((int(a), g, 0, 0), (seed, 0))
            for j in range(4):
                m = 4 * g + j
                if m < M:
                    out[m, i] = amp * (2.0 * ((w[j] >> 11) * 2.0 ** -53) - 1.0)
    return out


def noise_gaussian(seed, cells, M, sigma) -> np.ndarray:
    """Zero-mean Gaussian epsilon [M][len(cells)] of standard deviation sigma
    (the Gaussian variant of the noise experiments, Sec. V-D): for global
    cell a and field m, words 2 (m % 2) and 2 (m % 2) + 1 of Philox4x64-10 at
    counter (a, m // 2, 1, 0) and key (seed, 0) give u1 = ((w1 >> 11) + 1/2)
    2^-53 in (0, 1) and u2 = (w2 >> 11) 2^-53, and epsilon = sigma
    sqrt(-2 ln u1) cos(2 pi u2) (Box and Muller, 1958).  The third counter word
    keeps this stream apart from the uniform one.  Plain loops: small cases
    only."""
    out = np.empty((M, len(cells)))
    for i, a in enumerate(cells):
        for g in range((M + 1) // 2):
            w = philox4x64_10((int(a), g, 1, 0), (seed, 0))
            for j in range(2):
                m = 2 * g + j
                if m < M:
                    u1 = ((w[2 * j] >> 11) + 0.5) * 2.0 ** -53
                    u2 = (w[2 * j + 1] >> 11) * 2.0 ** -53
                    out[m, i] = sigma * np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return out


def apply_operator(A, T) -> np.ndarray:
    """q [M][n]: q_m = A T_m for every field."""
    T = np.asarray(T, np.float64)
    return (A @ T.T).T.copy()


def pair_errors(A, U_ref, C, T, q):
    """Per-field relative L2 errors of generated pairs (T_m, q_m).

    e_T    = ||T_m - (U_ref C)_m|| / ||(U_ref C)_m||
    e_q    = ||q_m - A (U_ref C)_m|| / ||A (U_ref C)_m||
    e_pair = ||A T_m - q_m|| / ||q_m||  (A applied to the field as stored)
    """
    T = np.asarray(T, np.float64)
    q = np.asarray(q, np.float64)
    T_ref = combine(U_ref, C)
    q_ref = apply_operator(A, T_ref)
    Aq = apply_operator(A, T)

    def rel(a, b):
        nb = np.linalg.norm(b, axis=1)
        return np.linalg.norm(a - b, axis=1) / np.where(nb > 0, nb, 1.0)

    return {"e_T": rel(T, T_ref), "e_q": rel(q, q_ref), "e_pair": rel(Aq, q)}


def generate(chip, density, C, rtol=1e-12, maxiter=100000, X0=None):
    """Whole hot path on one chip: assemble, block solve, combine, apply."""
    A = assemble(chip)
    B = rhs(chip, density)
    U, info = block_cg(A, B, X0=X0, rtol=rtol, maxiter=maxiter)
    T = combine(U, C)
    q = apply_operator(A, T)
    return {"A": A, "B": B, "U": U, "T": T, "q": q, "info": info}
