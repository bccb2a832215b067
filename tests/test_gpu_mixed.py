"""Parity of the tensor-core path (EWALD_MIXED: FP32 pairs, split-FP16 tcgen05 products
with FP32 accumulation, FP64 reductions) against the FP64 CPU oracle.

Bound: relative RMS force error and relative energy error <= 1e-5 against the oracle at
the same (beta, r_c, k_max).  The split-FP16 operands carry ~2^-22 relative error per term
and the phases ~4e-7 absolute (32-bit fixed-point angle, hardware sincos), so the observed
error is expected near 1e-7..1e-6.  EWALD_MIXED_BF16 keeps 8 fewer mantissa bits per term
(~2^-17 per product): bound 2e-4.
"""
import numpy as np
import pytest

from gpu_common import dev, mode_scale, need_gpu, oracle_cached, rel, rel_rms, rel_total, assert_close, torch

import oracle
from paper_1708_01135_gb300 import Ewald, PART_REAL, PART_RECIP, PART_SELF, tune
from paper_1708_01135_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _run(ew, pos, q, parts):
    n = len(q)
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    e = torch.empty(4, dtype=torch.float64, device="cuda")
    ew.compute_async(dev(pos), dev(q), F, e, parts=parts)
    assert ew.status() == 0
    return F.cpu().numpy(), e.cpu().numpy()


def test_unjittered_lattice_structure_factor():
    need_gpu()
    pos, q, L = W.rocksalt(8)
    with Ewald(L, 1.0, 4.0, 8, "mixed") as ew:
        _run(ew, pos, q, PART_RECIP)
        m = ew.kset()
        S = ew.structure_factor()
    hit = np.all((m % 8) == 4, axis=1)
    assert hit.sum() == 4
    assert np.abs(S[hit] - len(q)).max() < 2e-3 * len(q) ** 0.5
    assert np.abs(S[~hit]).max() < 2e-3 * len(q) ** 0.5


@pytest.mark.parametrize("case", [("rocksalt_512", 1.0, 4.0, 10), ("rocksalt_512", 1.3, 2.6, 8)])
def test_parts_match_oracle(case):
    need_gpu()
    name, beta, rc, kmax = case
    pos, q, L = getattr(W, name)()
    ref = oracle_cached(name, beta, rc, kmax)
    with Ewald(L, beta, rc, kmax, "mixed") as ew:
        Fk, ek = _run(ew, pos, q, PART_RECIP)
        m = ew.kset()
        S = ew.structure_factor()
        Fa, ea = _run(ew, pos, q, PART_REAL | PART_RECIP | PART_SELF)
    assert np.array_equal(m, ref["m"])
    assert np.all(np.abs(S - ref["S"]) < 1e-5 * mode_scale(q, m, ref["S"]))
    assert_close(Fk, ref["F_recip"], 1e-5)
    assert rel(ek[1], ref["E_recip"]) < 1e-5
    assert_close(Fa, ref["F"], 1e-5)
    assert rel(ea[3], ref["E_total"]) < 1e-5


@pytest.mark.parametrize("n,seed", [(4002, 77), (1030, 3)])
def test_random_systems_ragged(n, seed):
    """Ragged particle counts (not multiples of the 128/256-particle tiles or the 64-particle
    stages) and mixed +-1/+-2 charges."""
    need_gpu()
    pos, q, L = W.random_neutral(n, density=1.0, hard_core=0.8, seed=seed,
                                 mix=((1.0, 0.4), (2.0, 0.1)))
    rc, beta, kmax = 0.45 * L, 0.85, 14
    ref = oracle.ewald(pos, q, L, beta, rc, kmax)
    with Ewald(L, beta, rc, kmax, "mixed") as ew:
        F, e = ew.compute(dev(pos), dev(q))
    assert_close(F.cpu().numpy(), ref["F"], 1e-5)
    assert rel_total(e[3], ref) < 1e-5


def test_large_kmax_two_column_passes():
    """k_max = 45: 3 (2 k_max + 1) = 273 back-scatter columns need two passes."""
    need_gpu()
    pos, q, L = W.random_neutral(2000, density=1.0, hard_core=0.8, seed=8)
    beta, rc, kmax = 1.6, 0.45 * L, 45
    ref = oracle.ewald(pos, q, L, beta, rc, kmax)
    with Ewald(L, beta, rc, kmax, "mixed") as ew:
        F, e = ew.compute(dev(pos), dev(q))
    assert_close(F.cpu().numpy(), ref["F"], 1e-5)
    assert rel_total(e[3], ref) < 1e-5


def test_bf16_split_variant():
    need_gpu()
    pos, q, L = W.rocksalt_512()
    ref = oracle_cached("rocksalt_512", 1.0, 4.0, 10)
    with Ewald(L, 1.0, 4.0, 10, "mixed_bf16") as ew:
        F, e = ew.compute(dev(pos), dev(q))
    assert_close(F.cpu().numpy(), ref["F"], 2e-4)
    assert rel(e[3], ref["E_total"]) < 2e-4


def test_mixed_is_deterministic():
    need_gpu()
    pos, q, L = W.random_neutral(3000, density=1.0, hard_core=0.8, seed=21)
    with Ewald(L, 0.9, 4.0, 16, "mixed") as ew:
        F1, e1 = ew.compute(dev(pos), dev(q))
        F2, e2 = ew.compute(dev(pos), dev(q))
    assert torch.equal(F1, F2) and np.array_equal(e1, e2)


def test_full_size_random_32768_sampled():
    """The benchmarked workload and launch configuration: N = 32,768, L = 32, r_c = 4,
    (beta, k_max) from the tuner for 1e-6.  The oracle evaluates S(k) from all particles and
    forces on 512 sampled particles; the total energy comes from the full oracle sums."""
    need_gpu()
    pos, q, L = W.random_32768()
    rc, beta, kmax = tune(len(q), L, 1e-6, r_c=4.0)
    rng = np.random.default_rng(11)
    sub = np.sort(rng.choice(len(q), 512, replace=False))
    ek, Fk, _, S, _ = oracle.recip(pos, q, L, beta, kmax, sub=sub)
    _, Fr, _ = oracle.real(pos, q, L, beta, rc, sub=sub)
    with Ewald(L, beta, rc, kmax, "mixed") as ew:
        F, e = ew.compute(dev(pos), dev(q))
        Sg = ew.structure_factor()
    F = F.cpu().numpy()[sub]
    assert_close(F, Fr + Fk, 1e-5)
    assert rel(e[1], ek) < 1e-5
    assert np.all(np.abs(Sg - S) < 1e-5 * mode_scale(q, oracle.kset_half(kmax), S))
