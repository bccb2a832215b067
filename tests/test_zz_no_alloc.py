"""The allocation-free real-space entry point (ewald_real_noalloc), for callers that cannot
allocate device memory (stream capture, foreign allocators, allocation-free loops).

It is checked through the C ABI against the plan-based entry point (an EWALD_FP64 plan
evaluated with EWALD_PART_REAL), within the FP64 tolerance used by the other FP64 parity
tests (1e-10 relative), on two calls in a row with different systems, so that a result that
depended on the previous call's scratch contents would show.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from gpu_common import dev, need_gpu, rel, rel_rms, assert_close, torch

from paper_1708_01135_gb300 import Ewald, PART_REAL
from paper_1708_01135_gb300 import ewald as E
from paper_1708_01135_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _plan_real(pos, q, L, beta, rc):
    n = len(q)
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    e = torch.empty(4, dtype=torch.float64, device="cuda")
    with Ewald(L, beta, rc, 4, "fp64") as ew:
        ew.compute_async(dev(pos), dev(q), F, e, parts=PART_REAL)
        assert ew.status() == 0
    return F.cpu().numpy(), e.cpu().numpy()


def _noalloc(pos, q, L, beta, rc):
    lib = E.lib()
    n = len(q)
    tp, tq = dev(pos), dev(q)
    F = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
    e = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream or None
    status = lib.ewald_real_noalloc(L, beta, rc, n, tp.data_ptr(), tq.data_ptr(), F.data_ptr(),
                                    e.data_ptr(), st)
    assert status == 0, E.strerror(status)
    torch.cuda.synchronize()
    return F.cpu().numpy(), e.cpu().numpy()


def test_noalloc_matches_plan_entry_point_on_two_calls():
    need_gpu()
    systems = [
        W.random_neutral(3000, density=1.0, hard_core=0.8, seed=31, mix=((1.0, 0.4), (2.0, 0.1))),
        W.rocksalt(8, 1.0, 0.05, seed=32),     # second call: fewer particles than the first
    ]
    for pos, q, L in systems:
        beta, rc = 0.95, min(4.0, 0.5 * L)
        F_ref, e_ref = _plan_real(pos, q, L, beta, rc)
        F, e = _noalloc(pos, q, L, beta, rc)
        assert_close(F, F_ref, TOL)
        assert rel(e[0], e_ref[0]) < TOL
        assert e[1] == 0.0 and e[2] == 0.0 and e[3] == e[0]


def test_noalloc_rejects_sizes_beyond_its_scratch():
    need_gpu()
    lib = E.lib()
    n = E.NOALLOC_MAX_N + 1
    tp = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    tq = torch.zeros(n, dtype=torch.float64, device="cuda")
    F = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    e = torch.zeros(4, dtype=torch.float64, device="cuda")
    status = lib.ewald_real_noalloc(40.0, 1.0, 4.0, n, tp.data_ptr(), tq.data_ptr(), F.data_ptr(),
                                    e.data_ptr(), None)
    assert status == E.E_UNSUPPORTED
