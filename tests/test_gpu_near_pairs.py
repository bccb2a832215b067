"""Near real-space Coulomb pairs in double-float arithmetic (ewald_set_near_pairs) against the
FP64 oracle on a jittered rock-salt crystal, where the net force on an ion is a small sum of
large pair forces (Eq. 4, Section 2; the crystal stands in for the paper's NaCl systems,
Section 4)."""
import numpy as np
import pytest

from gpu_common import dev, need_gpu, rel_rms, assert_close

import oracle
from paper_1708_01135_gb300 import Ewald, PART_REAL
from paper_1708_01135_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# 16^3 ions, r_c = 4: cell mode (12 cells per side, stencil half-width 3) with four warps per
# group of targets; 44^3 ions: two warps per group (one warp per group: the 262,144-ion crystal
# of test_gpu_large.py)
CASES = [(16, 0.93, 4.0, 11), (44, 0.80, 4.8, 13)]


def _real(ew, pos, q, n):
    import torch
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    e = torch.empty(4, dtype=torch.float64, device="cuda")
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    ew.compute_phi_async(dev(pos), dev(q), F, phi, e, parts=PART_REAL)
    assert ew.status() == 0
    return F.cpu().numpy(), e.cpu().numpy(), phi.cpu().numpy()


@pytest.mark.parametrize("m,beta,rc,seed", CASES)
def test_double_float_near_pairs_match_the_oracle(m, beta, rc, seed):
    need_gpu()
    pos, q, L = W.rocksalt(m, a=1.0, jitter=0.05, seed=seed)
    n = len(q)
    e_ref, F_ref, phi_ref = oracle.real_cells(pos, q, L, beta, rc)
    with Ewald(L, beta, rc, 8, "mixed") as ew:
        F32, e32, phi32 = _real(ew, pos, q, n)
        assert ew.info()["stencil"] > 0          # the cell kernel, not the all-pairs one
        ew.set_near_pairs(True)
        Fdf, edf, phidf = _real(ew, pos, q, n)
        Fdf2, _, _ = _real(ew, pos, q, n)
        ew.set_near_pairs(False)
        F32b, _, _ = _real(ew, pos, q, n)
    err32, errdf = rel_rms(F32, F_ref), rel_rms(Fdf, F_ref)
    # the double-float near pairs: an order of magnitude below the FP32 ones on the crystal
    assert_close(Fdf, F_ref, 1e-7)
    assert errdf < 0.3 * err32, (errdf, err32)
    assert_close(phidf, phi_ref, 1e-7)
    # E_real: the erfc fit's error (below 7.6e-9 relative, systematic in r) adds up over the
    # pairs, so the bound is on the scale 1/2 sum |q_i phi_i| with a margin over the fit
    assert abs(edf[0] - e_ref) <= 2e-8 * 0.5 * np.abs(q * phi_ref).sum()
    # deterministic, and switching back restores the FP32 results bit for bit
    assert np.array_equal(Fdf, Fdf2)
    assert np.array_equal(F32, F32b)
