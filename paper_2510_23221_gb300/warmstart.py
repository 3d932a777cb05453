"""Learned warm start of block CG with the Fourier neural operator (fno.py).

    python -m paper_2510_23221_gb300.warmstart --train-chips 128 --eval-chips 512 --epochs 12

Data: chips of the benchmark chip's distribution (128x128x8, 8 layers, k
log-uniform in [1, 400], s = 32 power maps) from the seeded training range;
their basis solutions come from this library's block CG (mixed precision,
Jacobi, relative residual 1e-6).  Each right-hand side is one sample:

  inputs  (5 channels per cell): (log10 k - 1.3) / 0.75, power density on the
          top layer divided by the sample's peak density (zero elsewhere),
          and the centred x, y, z cell coordinates;
  target  theta / q_peak * t_scale (the solution is linear in the power
          map, so the network learns the response to a unit-peak map;
          t_scale makes targets of order one).

Training minimises the mean squared error with Adam (cosine learning rate)
entirely in the library's kernels; PyTorch only holds device memory and
shuffles sample indices.  Evaluation on held-out chips (disjoint seeds):
predict U (network outputs scaled back into the basis by
blockoa_fno_basis), measure its relative residual ||B_j - A U_j|| / ||B_j||
(blockoa_residual_ratio), warm-start block CG with the prediction when
every column's residual is <= the fallback threshold (1e-2) and from zero
otherwise, and compare iterations and time to 1e-6 with the zero start.
The solver is the benchmark's chosen form (pipeline.CHOSEN_SOLVE) unless
another is given.
"""
from __future__ import annotations

import argparse
import json
import math
import statistics
import time

import numpy as np

from . import blockoa as bo
from . import fno, pipeline, synth

LOGK_MEAN, LOGK_STD = 1.3, 0.75
C_IN = 5


def features(chip, dens) -> tuple:
    """(inputs float32 [s][nz][ny][nx][5], peak density float64 [s])."""
    s = dens.shape[0]
    nz, ny, nx = chip.nz, chip.ny, chip.nx
    X = np.zeros((s, nz, ny, nx, C_IN), np.float32)
    X[..., 0] = ((np.log10(chip.cell_k()) - LOGK_MEAN) / LOGK_STD)[None]
    qpk = np.abs(dens).reshape(s, -1).max(axis=1)
    qpk = np.where(qpk > 0, qpk, 1.0)
    X[:, 0, :, :, 1] = dens / qpk[:, None, None]
    X[..., 2] = (np.arange(nx) / max(nx - 1, 1) - 0.5)[None, None, None, :]
    X[..., 3] = (np.arange(ny) / max(ny - 1, 1) - 0.5)[None, None, :, None]
    X[..., 4] = (np.arange(nz) / max(nz - 1, 1) - 0.5)[None, :, None, None]
    return X, qpk


def solve(op, B, s, x0=None, rtol=1e-6, solve_kw=None):
    """Block CG (the chosen form unless solve_kw says otherwise); returns
    (U, stats, milliseconds)."""
    import torch
    kw = dict(pipeline.CHOSEN_SOLVE if solve_kw is None else solve_kw)
    U = torch.empty_like(B)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    st = bo.block_solve(op, B, U, s, rtol=rtol, x0=x0, raise_on_error=False, **kw)
    e1.record()
    torch.cuda.synchronize()
    return U, st, e0.elapsed_time(e1)


def relres(op, U, B, s):
    """||B_j - A U_j|| / ||B_j|| per column (blockoa_residual_ratio, float64)."""
    import torch
    r = torch.empty(op.n_chips * s, dtype=torch.float64, device="cuda")
    bo.residual_ratio(op, B, U, s, r)
    return r.cpu().numpy()


def shape_for(chip, max_batch=8, **kw) -> fno.FnoShape:
    return fno.FnoShape(nx=chip.nx, ny=chip.ny, nz=chip.nz, c_in=C_IN, max_batch=max_batch, **kw)


def init_params(shape: fno.FnoShape, seed: int) -> np.ndarray:
    """Seeded uniform fan-in initialisation (spectral weights 1 / width^2)."""
    rng = np.random.default_rng(seed)
    W, L, M, H = shape.width, shape.layers, shape.mx * shape.my * shape.mz, shape.hidden
    lim = lambda fan_in: 1.0 / math.sqrt(fan_in)
    parts = {
        "P": rng.uniform(-lim(shape.c_in), lim(shape.c_in), (W, shape.c_in)), "bP": np.zeros(W),
        "Wl": rng.uniform(-lim(W), lim(W), (L, W, W)), "bl": np.zeros((L, W)),
        "Rr": rng.uniform(0.0, 1.0, (L, M, W, W)) / (W * W), "Ri": rng.uniform(0.0, 1.0, (L, M, W, W)) / (W * W),
        "Q1": rng.uniform(-lim(W), lim(W), (H, W)), "c1": np.zeros(H),
        "Q2": rng.uniform(-lim(H), lim(H), (1, H)), "c2": np.zeros(1),
    }
    return fno.pack(parts, L)


class WarmStart:
    """A trained network and the target scale it was trained with."""

    def __init__(self, net: fno.Fno, t_scale: float):
        self.net, self.t_scale = net, t_scale

    def predict(self, op, chip, dens):
        """Predicted basis U [n][s] (float64 device tensor) of the one-chip
        operator op, and the milliseconds of the network and the scaling."""
        import torch
        X, qpk = features(chip, dens)
        s = X.shape[0]
        Xd = torch.from_numpy(X).cuda()
        Y = torch.empty((s, chip.nz, chip.ny, chip.nx), dtype=torch.float32, device="cuda")
        scale = torch.from_numpy(qpk / self.t_scale).cuda()
        U = torch.empty(op.n_total * s, dtype=torch.float64, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mb = self.net.shape.max_batch
        for b0 in range(0, s, mb):
            b1 = min(s, b0 + mb)
            self.net.forward(Xd[b0:b1], Y[b0:b1], b1 - b0)
        fno.basis(op, Y, scale, s, U)
        e1.record()
        torch.cuda.synchronize()
        return U, e0.elapsed_time(e1)


def build_dataset(seeds, nx=128, ny=128, n_layers=8, s=32, t_scale=None):
    """Device tensors X [S][nz][ny][nx][5], Y [S][nz][ny][nx], the target scale and solve stats."""
    import torch
    Xs, Ys, iters = [], [], []
    for seed in seeds:
        chip, dens = synth.warm_start_chip(seed, nx, ny, n_layers, s)
        op = bo.assemble([chip])
        B = torch.empty(op.n_total * s, dtype=torch.float64, device="cuda")
        bo.build_rhs(op, torch.from_numpy(np.ascontiguousarray(dens.ravel())).cuda(), B, s)
        U, st, _ = solve(op, B, s)
        iters.append(st[0].iters)
        X, qpk = features(chip, dens)
        theta = U.view(op.n_total, s).t().cpu().numpy() / qpk[:, None]     # [s][n]
        if t_scale is None:
            t_scale = 1.0 / float(np.mean(np.abs(theta)))
        Xs.append(torch.from_numpy(X).cuda())
        Ys.append(torch.from_numpy((theta * t_scale).astype(np.float32).reshape(s, chip.nz, chip.ny, chip.nx)).cuda())
        op.close()
    return torch.cat(Xs), torch.cat(Ys), t_scale, iters


def train(net: fno.Fno, X, Y, epochs: int, lr: float, seed: int = 0, log=None):
    """Adam with a cosine learning rate over epochs x batches; returns per-epoch mean losses."""
    import torch
    S = X.shape[0]
    mb = net.shape.max_batch
    g = torch.Generator().manual_seed(seed)
    steps = epochs * ((S + mb - 1) // mb)
    yb = torch.empty((mb,) + tuple(Y.shape[1:]), dtype=torch.float32, device="cuda")
    dy = torch.empty_like(yb)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    t, hist = 0, []
    for ep in range(epochs):
        perm = torch.randperm(S, generator=g)
        tot = 0.0
        for b0 in range(0, S, mb):
            idx = perm[b0:b0 + mb].cuda()
            nb = idx.numel()
            xb = X.index_select(0, idx).contiguous()
            tb = Y.index_select(0, idx).contiguous()
            net.zero_grad()
            net.forward(xb, yb[:nb], nb, keep=True)
            net.mse(yb[:nb], tb, nb, dy[:nb], loss)
            net.backward(dy[:nb], nb)
            t += 1
            net.adam_step(lr * 0.5 * (1.0 + math.cos(math.pi * (t - 1) / steps)), t)
            tot += loss.item() * nb
        hist.append(tot / S)
        if log:
            log(f"epoch {ep + 1}/{epochs} loss {hist[-1]:.5f}")
    return hist


def evaluate(ws: WarmStart, seeds, threshold=1e-2, nx=128, ny=128, n_layers=8, s=32, solve_kw=None):
    """Zero start vs learned start (with fallback) on held-out chips."""
    import torch
    rows = []
    for seed in seeds:
        chip, dens = synth.warm_start_chip(seed, nx, ny, n_layers, s)
        op = bo.assemble([chip])
        B = torch.empty(op.n_total * s, dtype=torch.float64, device="cuda")
        bo.build_rhs(op, torch.from_numpy(np.ascontiguousarray(dens.ravel())).cuda(), B, s)
        solve(op, B, s, solve_kw=solve_kw)   # warm-up: workspace and graph of this operator
        U0, st0, ms0 = solve(op, B, s, solve_kw=solve_kw)
        U_pred, ms_pred = ws.predict(op, chip, dens)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rr = relres(op, U_pred, B, s)
        e1.record()
        torch.cuda.synchronize()
        ms_check = e0.elapsed_time(e1)
        warm = bool(np.max(rr) <= threshold)
        _, st1, ms1 = solve(op, B, s, x0=U_pred, solve_kw=solve_kw)
        # the zero-start basis (relative residual 1e-6) is the reference for the prediction's error
        u0, up = U0.cpu().numpy(), U_pred.cpu().numpy()
        err = float(np.linalg.norm(up - u0) / np.linalg.norm(u0))
        rows.append({"seed": seed, "zero_iters": st0[0].iters, "zero_ms": ms0,
                     "warm_iters": st1[0].iters, "warm_ms": ms1, "pred_ms": ms_pred, "check_ms": ms_check,
                     "pred_relres_max": float(np.max(rr)), "pred_relres_median": float(np.median(rr)),
                     "pred_rel_error": err, "use_warm": warm,
                     "ok": st0[0].status == bo.OK and st1[0].status == bo.OK})
        op.close()
    chosen_iters = [r["warm_iters"] if r["use_warm"] else r["zero_iters"] for r in rows]
    chosen_ms = [r["pred_ms"] + r["check_ms"] + (r["warm_ms"] if r["use_warm"] else r["zero_ms"]) for r in rows]
    return {
        "rows": rows, "chips": len(rows), "threshold": threshold,
        "warm_start_used": sum(r["use_warm"] for r in rows),
        "zero_iters_mean": statistics.mean(r["zero_iters"] for r in rows),
        "zero_iters_median": statistics.median(r["zero_iters"] for r in rows),
        "chosen_iters_mean": statistics.mean(chosen_iters),
        "chosen_iters_median": statistics.median(chosen_iters),
        "always_warm_iters_mean": statistics.mean(r["warm_iters"] for r in rows),
        "zero_ms_mean": statistics.mean(r["zero_ms"] for r in rows),
        "zero_ms_median": statistics.median(r["zero_ms"] for r in rows),
        "chosen_ms_mean": statistics.mean(chosen_ms),
        "chosen_ms_median": statistics.median(chosen_ms),
        "always_warm_ms_mean": statistics.mean(r["pred_ms"] + r["warm_ms"] for r in rows),
        "pred_ms_mean": statistics.mean(r["pred_ms"] for r in rows),
        "pred_relres_median": statistics.median(r["pred_relres_median"] for r in rows),
        "pred_relres_max_median": statistics.median(r["pred_relres_max"] for r in rows),
        "pred_rel_error_median": statistics.median(r["pred_rel_error"] for r in rows),
        "all_converged": all(r["ok"] for r in rows),
    }


def main():
    import torch
    from . import build
    p = argparse.ArgumentParser()
    p.add_argument("--train-chips", type=int, default=128)
    p.add_argument("--eval-chips", type=int, default=512)
    p.add_argument("--epochs", type=int, default=12)
    p.add_argument("--batch", type=int, default=8)
    p.add_argument("--lr", type=float, default=2e-3)
    p.add_argument("--threshold", type=float, default=1e-2)
    p.add_argument("--nx", type=int, default=128)
    p.add_argument("--layers", type=int, default=4)
    a = p.parse_args()
    build.build()
    t0 = time.perf_counter()
    tr_seeds = [synth.FNO_TRAIN_SEED0 + i for i in range(a.train_chips)]
    X, Y, t_scale, tr_iters = build_dataset(tr_seeds, nx=a.nx, ny=a.nx)
    t_data = time.perf_counter() - t0
    chip0, _ = synth.warm_start_chip(tr_seeds[0], a.nx, a.nx)
    shape = shape_for(chip0, max_batch=a.batch, layers=a.layers)
    net = fno.Fno(shape, init_params(shape, 1234))
    t1 = time.perf_counter()
    hist = train(net, X, Y, a.epochs, a.lr, log=lambda m: print(m, flush=True))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    del X, Y
    ws = WarmStart(net, t_scale)
    ev = evaluate(ws, [synth.FNO_HELDOUT_SEED0 + i for i in range(a.eval_chips)], a.threshold, nx=a.nx, ny=a.nx)
    print(json.dumps({"network": {"nx": shape.nx, "ny": shape.ny, "nz": shape.nz, "width": shape.width,
                                  "layers": shape.layers, "modes": [shape.mx, shape.my, shape.mz],
                                  "params": net.n_params},
                      "train": {"chips": a.train_chips, "samples": a.train_chips * 32, "epochs": a.epochs,
                                "batch": a.batch, "lr": a.lr, "loss_first": hist[0], "loss_last": hist[-1],
                                "data_s": round(t_data, 1), "train_s": round(t_train, 1),
                                "solve_iters_mean": statistics.mean(tr_iters)},
                      "eval": {k: v for k, v in ev.items() if k != "rows"}}), flush=True)


if __name__ == "__main__":
    main()
