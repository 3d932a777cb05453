"""The allocation-free pair check agrees with the allocating one.

blockoa_pair_check_static is for callers that cannot allocate device memory
while they run (memory reserved up front by their own pool, a fixed budget
that forbids allocation after start-up, or a loop that must not stall on
cudaMalloc / cudaFree).  It keeps its accumulators in a fixed device array
shared by all calls, so two calls in a row must both give the same result
as blockoa_pair_check: the second call proves the array is cleared.  After
a first call (which looks up the array's address and loads the kernels),
the device's free memory must not shrink across further calls.
"""
import ctypes as ct

import numpy as np
import pytest
import torch

from paper_2510_23221_gb300 import blockoa as bo
from paper_2510_23221_gb300 import build as bld
from paper_2510_23221_gb300 import synth

pytestmark = pytest.mark.gpu


def _static_entry():
    bld.build()
    lib = bo.library()
    fn = lib.blockoa_pair_check_static
    fn.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_int, ct.c_void_p,
                   ct.c_void_p]
    fn.restype = ct.c_int
    return fn


@pytest.mark.parametrize("dtype", [bo.FP64, bo.MIXED])
def test_static_pair_check_matches_allocating_check_twice(dtype):
    fn = _static_entry()
    chips = [synth.reference_stack_chip(), synth.random_small_chip(7, 21, 13, 3)]
    op = bo.assemble(chips)
    M = 12
    tdt = torch.float64 if dtype == bo.FP64 else torch.float32
    rng = np.random.default_rng(3)
    T = torch.from_numpy(rng.standard_normal(op.n_total * M)).to(tdt).cuda()
    q = torch.empty_like(T)
    bo.apply_operator(op, T, q, M, dtype)
    # perturb every field by a different amount so each e_pair differs
    for c in range(op.n_chips):
        sz = op.sizes[c]
        view = q[sz["off"] * M:(sz["off"] + sz["n"]) * M].view(M, sz["n"])
        view *= (1 + 1e-6 * torch.arange(1, M + 1, dtype=tdt, device="cuda"))[:, None]
    ref = torch.empty(op.n_chips * M, dtype=torch.float64, device="cuda")
    bo.pair_check(op, T, q, M, dtype, ref)
    expect = ref.cpu().numpy()
    assert np.all(expect > 1e-8)
    stream = torch.cuda.current_stream().cuda_stream
    first = torch.full_like(ref, float("nan"))
    assert fn(op.handle, T.data_ptr(), q.data_ptr(), M, dtype, first.data_ptr(), stream) == bo.OK
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        out = torch.full_like(ref, float("nan"))
        rc = fn(op.handle, T.data_ptr(), q.data_ptr(), M, dtype, out.data_ptr(), stream)
        assert rc == bo.OK, bo.status_string(rc)
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), expect, rtol=1e-12, atol=0)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free_before


def test_static_pair_check_rejects_sizes_beyond_its_array():
    fn = _static_entry()
    op = bo.assemble([synth.random_small_chip(8, 4, 4, 2), synth.random_small_chip(9, 4, 4, 2)])
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    M = 20000   # 2 chips x 20000 fields > BLOCKOA_STATIC_PAIR_MAX; rejected before any launch
    rc = fn(op.handle, buf.data_ptr(), buf.data_ptr(), M, bo.FP64, buf.data_ptr(), None)
    assert rc == bo.ERR_INVALID
    assert b"BLOCKOA_STATIC_PAIR_MAX" in bo.library().blockoa_last_error()
