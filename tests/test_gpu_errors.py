"""Edge cases and error statuses of the C ABI on the GPU: empty input, tiny systems,
non-neutral and non-finite input reported as status codes, and the paper's degenerate
cases (a single neutral pair, r_c = L/2 exactly on a lattice), and the timeout path of the
bounded device waits."""
import math

import numpy as np
import pytest

from gpu_common import dev, need_gpu, rel, rel_rms, assert_close, torch

import oracle
from paper_1708_01135_gb300 import Ewald, EwaldError
from paper_1708_01135_gb300 import ewald as E
from paper_1708_01135_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_empty_input_gives_zero_energy(prec):
    need_gpu()
    with Ewald(8.0, 1.0, 4.0, 8, prec) as ew:
        F, e = ew.compute(torch.zeros((0, 3), dtype=torch.float64, device="cuda"),
                          torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert F.shape == (0, 3) and np.all(e == 0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_single_pair(prec):
    need_gpu()
    L = 6.0
    pos = np.array([[1.0, 2.0, 3.0], [2.1, 2.4, 2.2]])
    q = np.array([1.5, -1.5])
    ref = oracle.ewald(pos, q, L, 1.1, 3.0, 9)
    with Ewald(L, 1.1, 3.0, 9, prec) as ew:
        F, e = ew.compute(dev(pos), dev(q))
    tol = 1e-10 if prec == "fp64" else 2e-5
    assert_close(F.cpu().numpy(), ref["F"], tol)
    assert rel(e[3], ref["E_total"]) < tol


def test_nonneutral_is_reported():
    need_gpu()
    pos, q, L = W.rocksalt_512()
    q = q.copy(); q[0] = 0.5
    with Ewald(L, 1.0, 4.0, 8, "fp64") as ew:
        with pytest.raises(EwaldError) as ex:
            ew.compute(dev(pos), dev(q))
        assert ex.value.status == E.E_NONNEUTRAL


def test_nonfinite_is_reported():
    need_gpu()
    pos, q, L = W.rocksalt_512()
    pos = pos.copy(); pos[3, 1] = np.nan
    with Ewald(L, 1.0, 4.0, 8, "fp64") as ew:
        with pytest.raises(EwaldError) as ex:
            ew.compute(dev(pos), dev(q))
        assert ex.value.status == E.E_NONFINITE
        # the plan stays usable after a reported error
        pos2, q2, _ = W.rocksalt_512()
        F, e = ew.compute(dev(pos2), dev(q2))
        assert math.isfinite(e[3])


def test_unjittered_lattice_at_half_box_cutoff():
    """r_c = L/2 on an exact lattice: pairs at exactly L/2 are excluded on both sides (strict
    inequality of Listing 1), so no image is counted twice."""
    need_gpu()
    pos, q, L = W.rocksalt(8)
    ref = oracle.ewald(pos, q, L, 1.0, 4.0, 10)
    with Ewald(L, 1.0, 4.0, 10, "fp64") as ew:
        F, e = ew.compute(dev(pos), dev(q))
    assert rel(e[0], ref["E_real"]) < 1e-12
    assert np.abs(F.cpu().numpy()).max() < 1e-10


def test_bounded_device_wait_times_out_and_the_device_stays_usable():
    """A device wait that can never complete (a barrier nothing arrives at, the way a staged
    copy that never landed would look) gives up after about a second and reports
    EWALD_E_TIMEOUT through the plan's status; the next evaluation on the same plan is
    correct, so the context survived."""
    need_gpu()
    import time
    pos, q, L = W.rocksalt_512()
    ref = oracle.ewald(pos, q, L, 1.0, 4.0, 10)
    with Ewald(L, 1.0, 4.0, 10, "mixed") as ew:
        t0 = time.perf_counter()
        ew.probe_timeout()
        st = ew.status()
        dt = time.perf_counter() - t0
        assert st == E.E_TIMEOUT
        assert 0.5 < dt < 60.0
        F, e = ew.compute(dev(pos), dev(q))
        assert ew.status() == 0
    assert_close(F.cpu().numpy(), ref["F"], 1e-5)
    assert rel(e[3], ref["E_total"]) < 1e-5
