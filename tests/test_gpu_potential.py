"""Per-particle potentials (ewald_compute_phi_async) against the oracle's phi_real and
phi_recip: phi_i = phi_i^real + phi_i^recip - 2 beta q_i / sqrt(pi), and the property
1/2 sum_i q_i phi_i = E_total, on every path (FP64, mixed, FP32) and for the part masks."""
import math

import numpy as np
import pytest

from gpu_common import dev, need_gpu, rel, rel_rms, assert_close, torch

import oracle
from paper_1708_01135_gb300 import PART_ALL, PART_REAL, PART_RECIP, PART_SELF, Ewald
from paper_1708_01135_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-5, "fp32": 1e-5}


def _run(ew, pos, q, parts=PART_ALL):
    n = len(q)
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    E = torch.empty(4, dtype=torch.float64, device="cuda")
    ew.compute_phi_async(dev(pos), dev(q), F, phi, E, parts=parts)
    assert ew.status() == 0
    return F.cpu().numpy(), phi.cpu().numpy(), E.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "mixed", "fp32"])
def test_potentials_match_oracle(precision):
    need_gpu()
    pos, q, L = W.random_neutral(4002, density=1.0, hard_core=0.8, seed=19,
                                 mix=((1.0, 0.4), (2.0, 0.1)))
    beta, rc, km = 0.85, 0.45 * L, 14
    ref = oracle.ewald(pos, q, L, beta, rc, km)
    phi_ref = ref["phi_real"] + ref["phi_recip"] - 2.0 * beta / math.sqrt(math.pi) * q
    with Ewald(L, beta, rc, km, precision) as ew:
        F, phi, E = _run(ew, pos, q)
        _, phr, _ = _run(ew, pos, q, PART_REAL)
        _, phk, _ = _run(ew, pos, q, PART_RECIP)
        _, phs, _ = _run(ew, pos, q, PART_SELF)
    tol = TOL[precision]
    assert_close(phr, ref["phi_real"], tol)
    assert_close(phk, ref["phi_recip"], tol)
    assert np.allclose(phs, -2.0 * beta / math.sqrt(math.pi) * q, rtol=1e-15, atol=0)
    assert_close(phi, phi_ref, tol)
    # the energy is half the charge-weighted sum of the potentials
    assert rel(0.5 * float((q * phi).sum()), E[3]) < max(tol, 1e-12)
    assert rel(0.5 * float((q * phi).sum()), ref["E_total"]) < tol


def test_potentials_on_a_rock_salt_lattice_equal_the_madelung_potential():
    """Unjittered rock-salt with unit spacing: every ion sits at the Madelung potential
    -q_i M_NaCl (r_0 = 1)."""
    need_gpu()
    pos, q, L = W.rocksalt(8)
    with Ewald(L, 1.0, 4.0, 10, "fp64") as ew:
        _, phi, _ = _run(ew, pos, q)
    M = 1.747564594633182
    assert np.abs(phi + q * M).max() < 1e-6
