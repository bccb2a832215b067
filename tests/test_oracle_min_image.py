"""Pins of the oracle's minimum-image branch of the real-space sum (Section 3.1.1, Eq. 4,
Listing 1), the branch every full-size parity test compares against (r_c <= L/2).

The Madelung, beta-invariance and brute-force pins of tests/test_oracle.py run at converged
cutoffs r_c > L/2, which take the explicit image loop.  Here, at r_c <= L/2:

* the minimum-image sum equals the image-loop sum over the 27 shifts |n_a| <= 1 (each pair
  term kept when its image lies within r_c), to rounding: the image loop is pinned by the
  Madelung constants and by brute-force lattice sums, so this carries those pins over;
* the minimum-image forces are the negative gradient of the minimum-image energy, by
  central differences on a 432-ion random system, with beta r_c = 5.6 so that a pair
  crossing the cutoff moves the energy by erfc(5.6) / r_c ~ 1e-15 only;
* the forces of the branch sum to zero (every pair adds equal and opposite forces).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1708_01135_gb300 import workloads as W


def _system():
    pos, q, L = W.random_neutral(432, density=1.0, hard_core=0.8, seed=4321,
                                 mix=((1.0, 0.4), (2.0, 0.1)))
    rc = 0.49 * L
    beta = 5.6 / rc
    return pos, q, L, beta, rc


@pytest.mark.parametrize("beta_rc", [5.6, 1.5])
def test_minimum_image_equals_image_loop(beta_rc):
    """At beta r_c = 1.5 the truncated tail erfc(1.5) ~ 3e-2 is large, so pairs near the
    cutoff matter and a wrong image choice or a non-strict cutoff test would show."""
    pos, q, L, _, rc = _system()
    beta = beta_rc / rc
    assert rc <= 0.5 * L
    e1, F1, p1 = O.real(pos, q, L, beta, rc)
    e2, F2, p2 = O.real(pos, q, L, beta, rc, images=True)
    assert abs(e1 - e2) <= 1e-12 * abs(e2)
    assert np.abs(F1 - F2).max() <= 1e-12 * np.abs(F2).max()
    assert np.abs(p1 - p2).max() <= 1e-12 * np.abs(p2).max()


def test_minimum_image_forces_are_energy_gradient():
    pos, q, L, beta, rc = _system()
    _, F, _ = O.real(pos, q, L, beta, rc)
    h = 1e-5
    rng = np.random.default_rng(7)
    picks = rng.choice(len(q), 12, replace=False)
    scale = math.sqrt(float((F ** 2).sum(axis=1).mean()))
    for i in picks:
        for a in range(3):
            p = pos.copy(); p[i, a] += h
            ep, _, _ = O.real(p, q, L, beta, rc)
            p[i, a] -= 2 * h
            em, _, _ = O.real(p, q, L, beta, rc)
            fd = -(ep - em) / (2 * h)
            assert abs(fd - F[i, a]) < 1e-6 * scale, (i, a, fd, F[i, a])


def test_minimum_image_forces_sum_to_zero():
    pos, q, L, beta, rc = _system()
    _, F, _ = O.real(pos, q, L, beta, rc)
    assert np.abs(F.sum(axis=0)).max() < 1e-11 * np.abs(F).sum()
