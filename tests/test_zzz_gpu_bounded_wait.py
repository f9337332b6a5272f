"""Failure detection on the GPU without a GPU fault: a bounded wait on a flag that nothing sets
runs out, the kernel reports HMPCG_E_TIMEOUT through device memory, and the context keeps
working afterwards."""
import time

import numpy as np
import pytest
import torch

import inputs
from oracle import grid

pytestmark = pytest.mark.gpu

h = pytest.importorskip("paper_2605_13343_gb300")


def test_bounded_wait_times_out_and_the_context_stays_usable():
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    h.selftest_wait(flag, status, 1 << 16)
    torch.cuda.synchronize()
    assert int(status.item()) == h.E_TIMEOUT
    assert time.perf_counter() - t0 < 10.0
    flag.fill_(1)
    h.selftest_wait(flag, status, 1 << 16)
    torch.cuda.synchronize()
    assert int(status.item()) == h.OK
    # the context still computes correctly after the timeout: an SpMV against the oracle
    fr = inputs.frame("disc2d_1024", 0)
    ref = grid.assemble(fr["rho"], fr["dims"])
    s = h.System(fr["dims"])
    h.assemble(torch.from_numpy(fr["rho"]).cuda(), s)
    xh = np.random.default_rng(0).standard_normal(1024).astype(np.float32)
    y = h.spmv(s, torch.from_numpy(xh).cuda(), torch.empty(1024, dtype=torch.float32, device="cuda"))
    want = grid.spmv(ref, xh.astype(np.float64))
    got = y.cpu().numpy().astype(np.float64)
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()
