"""Parity of the CUDA path against the FP64 CPU oracle, element by element, on the same
seeded inputs and the same (beta, r_c, k_max).

Tolerances (relative RMS over all force components, relative energy error):
  * EWALD_FP64 (FP64 CUDA cores): 1e-10.  The two sides differ only in summation order,
    the FP64 phase recurrence (error ~k_max * 1e-16) and erfc/exp rounding.
  * EWALD_FP32 (FP32 CUDA cores): 2e-5.  FP32 pair arithmetic on cell-local coordinates
    (~1e-7 per pair) and FP32 products of FP64-accurate phase tables summed over N.
  * EWALD_MIXED (tensor cores, split FP16): 1e-5, the mixed-path bound.
Each part (real, reciprocal, self) is compared separately as well as the total.
"""
import numpy as np
import pytest

from gpu_common import dev, mode_scale, need_gpu, oracle_cached, rel, rel_rms, assert_close, torch

import oracle
from paper_1708_01135_gb300 import Ewald, PART_REAL, PART_RECIP, PART_SELF
from paper_1708_01135_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-5, "mixed": 1e-5}


def _run(ew, pos, q, parts):
    n = len(q)
    tp, tq = dev(pos), dev(q)
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    e = torch.empty(4, dtype=torch.float64, device="cuda")
    ew.compute_async(tp, tq, F, e, parts=parts)
    assert ew.status() == 0
    return F.cpu().numpy(), e.cpu().numpy()


CASES = [
    # name, beta, rc, kmax
    ("rocksalt_512", 1.0, 4.0, 10),      # r_c = L/2: all-pairs minimum-image mode
    ("rocksalt_512", 1.3, 2.6, 8),       # cell mode, w = 1 (3 cells per side)
]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES)
def test_parts_match_oracle(prec, case):
    need_gpu()
    name, beta, rc, kmax = case
    pos, q, L = getattr(W, name)()
    ref = oracle_cached(name, beta, rc, kmax)
    tol = TOL[prec]
    with Ewald(L, beta, rc, kmax, prec) as ew:
        Fr, er = _run(ew, pos, q, PART_REAL)
        Fk, ek = _run(ew, pos, q, PART_RECIP)
        Fa, ea = _run(ew, pos, q, PART_REAL | PART_RECIP | PART_SELF)
    assert_close(Fr, ref["F_real"], tol)
    assert_close(Fk, ref["F_recip"], tol)
    assert_close(Fa, ref["F"], tol)
    assert rel(er[0], ref["E_real"]) < tol and er[1] == 0 and er[2] == 0
    assert rel(ek[1], ref["E_recip"]) < tol and ek[0] == 0
    assert rel(ea[2], ref["E_self"]) < 1e-14
    assert rel(ea[3], ref["E_total"]) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_structure_factor_per_mode(prec):
    need_gpu()
    pos, q, L = W.rocksalt_512()
    beta, rc, kmax = 1.0, 4.0, 10
    ref = oracle_cached("rocksalt_512", beta, rc, kmax)
    with Ewald(L, beta, rc, kmax, prec) as ew:
        _run(ew, pos, q, PART_RECIP)
        m = ew.kset()
        S = ew.structure_factor()
    assert np.array_equal(m, ref["m"])          # same K_half, same order
    tol = 1e-12 if prec == "fp64" else 2e-6
    assert np.all(np.abs(S - ref["S"]) < tol * mode_scale(q, m, ref["S"]))


def test_unjittered_lattice_structure_factor_is_exact():
    need_gpu()
    pos, q, L = W.rocksalt(8)
    with Ewald(L, 1.0, 4.0, 8, "fp64") as ew:
        _run(ew, pos, q, PART_RECIP)
        m = ew.kset()
        S = ew.structure_factor()
    hit = np.all((m % 8) == 4, axis=1)
    assert hit.sum() == 4
    assert np.allclose(S[hit], len(q), atol=1e-9)
    assert np.abs(S[~hit]).max() < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_random_system_multi_tile(prec):
    """A random ionic system spanning many cells, tiles and particle chunks, with a ragged
    tail (N not a multiple of 32 or of the block sizes)."""
    need_gpu()
    pos, q, L = W.random_neutral(4002, density=1.0, hard_core=0.8, seed=77,
                                 mix=((1.0, 0.4), (2.0, 0.1)))
    beta, rc, kmax = 0.9, 4.0, 18
    ref = oracle.ewald(pos, q, L, beta, rc, kmax)
    with Ewald(L, beta, rc, kmax, prec) as ew:
        info = ew.info()
        assert info["stencil"] == 2 and info["cells_per_side"] >= 5
        F, e = ew.compute(dev(pos), dev(q))
    F = F.cpu().numpy()
    tol = TOL[prec]
    assert_close(F, ref["F"], tol)
    assert rel(e[3], ref["E_total"]) < tol


def test_fp64_is_deterministic_and_wraps_positions():
    need_gpu()
    pos, q, L = W.random_neutral(1000, density=1.0, hard_core=0.8, seed=5)
    with Ewald(L, 0.9, 4.0, 12, "fp64") as ew:
        F1, e1 = ew.compute(dev(pos), dev(q))
        F2, e2 = ew.compute(dev(pos), dev(q))
        shifted = pos + L * np.array([3.0, -1.0, 2.0])
        F3, e3 = ew.compute(dev(shifted), dev(q))
    assert torch.equal(F1, F2) and np.array_equal(e1, e2)
    assert_close(F3.cpu().numpy(), F1.cpu().numpy(), 1e-12)
    assert rel(e3[3], e1[3]) < 1e-12


def test_workspace_grows_and_shrinks():
    need_gpu()
    with Ewald(10.0, 1.0, 3.0, 8, "fp64") as ew:
        for n, seed in ((200, 1), (800, 2), (100, 3)):
            pos, q, L = W.random_neutral(n, L=10.0, hard_core=0.5, seed=seed)
            ref = oracle.ewald(pos, q, L, 1.0, 3.0, 8)
            F, e = ew.compute(dev(pos), dev(q))
            assert_close(F.cpu().numpy(), ref["F"], 1e-10)
            assert rel(e[3], ref["E_total"]) < 1e-10


def test_host_buffer_entry_point():
    need_gpu()
    pos, q, L = W.rocksalt_512()
    ref = oracle_cached("rocksalt_512", 1.0, 4.0, 10)
    with Ewald(L, 1.0, 4.0, 10, "fp64") as ew:
        F, e = ew.compute_host(pos, q)
    assert_close(F, ref["F"], 1e-10)
    assert rel(e[3], ref["E_total"]) < 1e-10
