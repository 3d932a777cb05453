"""GPU parity of the warm-start Fourier neural operator against the float64
reference (oracle/fno_oracle.py): forward, every parameter gradient, loss
and Adam, through the C ABI.  The GPU multiplies by bfloat16 copies of the
weight matrices (biases stay float32), so the reference is given the same
rounded weights; the remaining difference is float32 arithmetic.
"""
import numpy as np
import pytest

from oracle import fno_oracle as fo

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WEIGHTS = ("P", "Wl", "Rr", "Ri", "Q1", "Q2")


def bf16(a):
    """Round float64 values to bfloat16 (nearest, ties to even), as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def setup(shape_kw, seed, batch=2):
    from paper_2510_23221_gb300 import fno
    sh = fo.FnoShape(**shape_kw)
    rng = np.random.default_rng(seed)
    p = fo.init_params(sh, seed)
    for k in p:
        p[k] = p[k] + 0.05 * rng.standard_normal(p[k].shape)
    flat = fno.pack(p, sh.layers)
    gshape = fno.FnoShape(nx=sh.nx, ny=sh.ny, nz=sh.nz, c_in=sh.c_in, width=sh.width, hidden=sh.hidden,
                          layers=sh.layers, mx=sh.mx, my=sh.my, mz=sh.mz, max_batch=batch)
    net = fno.Fno(gshape, flat)
    # the reference sees exactly the float32 parameters, weights rounded to bfloat16
    pf = fno.unpack(flat.astype(np.float64), fo.param_shapes(sh))
    ref = {k: (bf16(v) if k in WEIGHTS else v) for k, v in pf.items()}
    x = rng.standard_normal((batch, sh.nz, sh.ny, sh.nx, sh.c_in)).astype(np.float32)
    return sh, net, ref, x, rng


SMALL = dict(nx=16, ny=12, nz=4, c_in=3, width=32, hidden=32, layers=2, mx=4, my=4, mz=2)
MEDIUM = dict(nx=32, ny=24, nz=8, c_in=5, width=32, hidden=64, layers=3, mx=12, my=12, mz=4)


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-30)


@pytest.mark.parametrize("kw", [SMALL, MEDIUM])
def test_forward_matches_reference(kw):
    sh, net, ref, x, _ = setup(kw, 1)
    B = x.shape[0]
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty((B, sh.nz, sh.ny, sh.nx), dtype=torch.float32, device="cuda")
    net.forward(xd, yd, B)
    y_ref, _ = fo.forward(ref, x.astype(np.float64), sh)
    assert rel(yd.cpu().numpy(), y_ref) < 2e-5


@pytest.mark.parametrize("kw", [SMALL, MEDIUM])
def test_gradients_match_reference(kw):
    from paper_2510_23221_gb300 import fno
    sh, net, ref, x, rng = setup(kw, 2)
    B = x.shape[0]
    dy = rng.standard_normal((B, sh.nz, sh.ny, sh.nx)).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty((B, sh.nz, sh.ny, sh.nx), dtype=torch.float32, device="cuda")
    net.zero_grad()
    net.forward(xd, yd, B, keep=True)
    net.backward(torch.from_numpy(dy).cuda(), B)
    g_gpu = fno.unpack(net.grads().astype(np.float64), fo.param_shapes(sh))
    _, cache = fo.forward(ref, x.astype(np.float64), sh)
    g_ref = fo.backward(ref, cache, dy.astype(np.float64), sh)
    for k in g_ref:
        assert rel(g_gpu[k], g_ref[k]) < 1e-4, (k, rel(g_gpu[k], g_ref[k]))
    # gradients accumulate until zeroed
    net.forward(xd, yd, B, keep=True)
    net.backward(torch.from_numpy(dy).cuda(), B)
    g2 = fno.unpack(net.grads().astype(np.float64), fo.param_shapes(sh))
    assert rel(g2["Q1"], 2 * g_ref["Q1"]) < 1e-4


def test_mse_and_adam_step_match_reference():
    from paper_2510_23221_gb300 import fno
    sh, net, ref, x, rng = setup(SMALL, 3)
    B = x.shape[0]
    target = rng.standard_normal((B, sh.nz, sh.ny, sh.nx)).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty((B, sh.nz, sh.ny, sh.nx), dtype=torch.float32, device="cuda")
    dy = torch.empty_like(yd)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    net.zero_grad()
    net.forward(xd, yd, B, keep=True)
    net.mse(yd, torch.from_numpy(target).cuda(), B, dy, loss)
    y = yd.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - fo.loss(y, target)) <= 1e-5 * fo.loss(y, target)
    assert np.allclose(dy.cpu().numpy(), 2 * (y - target) / y.size, rtol=1e-5, atol=1e-12)
    net.backward(dy, B)
    p0 = net.params().astype(np.float64)
    g = net.grads().astype(np.float64)
    net.adam_step(lr=1e-3, t=1)
    P = {"w": p0.copy()}
    fo.adam_step(P, {"w": g}, {"w": np.zeros_like(g)}, {"w": np.zeros_like(g)}, t=1, lr=1e-3)
    assert np.allclose(net.params(), P["w"], rtol=0, atol=1e-6)


def test_training_steps_reduce_the_loss():
    sh, net, ref, x, rng = setup(SMALL, 4, batch=2)
    B = x.shape[0]
    # a learnable target: the reference network with other weights
    other = fo.init_params(sh, 99)
    t_ref, _ = fo.forward(other, x.astype(np.float64), sh)
    xd = torch.from_numpy(x).cuda()
    td = torch.from_numpy(t_ref.astype(np.float32)).cuda()
    yd = torch.empty_like(td)
    dy = torch.empty_like(td)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    losses = []
    for t in range(1, 61):
        net.zero_grad()
        net.forward(xd, yd, B, keep=True)
        net.mse(yd, td, B, dy, loss)
        losses.append(loss.item())
        net.backward(dy, B)
        net.adam_step(lr=3e-3, t=t)
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])


def test_invalid_arguments_rejected():
    from paper_2510_23221_gb300 import blockoa as bo
    from paper_2510_23221_gb300 import fno
    sh = fno.FnoShape(nx=16, ny=12, nz=4, c_in=3, hidden=32, layers=2, mx=4, my=4, mz=2, max_batch=1)
    with pytest.raises(bo.BlockoaError):
        fno.param_count(fno.FnoShape(nx=16, ny=12, nz=4, width=16))      # width must be 32
    with pytest.raises(bo.BlockoaError):
        fno.param_count(fno.FnoShape(nx=4, ny=12, nz=4, mx=12))          # more modes than cells
    net = fno.Fno(sh, np.zeros(fno.param_count(sh), np.float32))
    xd = torch.zeros((2, 4, 12, 16, 3), dtype=torch.float32, device="cuda")
    yd = torch.zeros((2, 4, 12, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(bo.BlockoaError):
        net.forward(xd, yd, 2)                                            # batch above max_batch
    with pytest.raises(bo.BlockoaError):
        net.backward(yd[:1], 1)                                           # no kept forward
    net.close()
