"""Pins of the SPME oracle (oracle/spme.py) against facts that fix it independently of its
own formulas:

* cardinal B-splines: partition of unity of M_p and of its derivative over integer shifts,
  symmetry about p/2, unit integral, the hat function at p = 2;
* convergence: as the mesh K and the order p grow, the SPME reciprocal energy, forces,
  potentials and virial converge to the classical Ewald reciprocal sum of ``oracle.recip``
  and ``oracle.virial_recip`` (themselves pinned in test_oracle*.py), down to rounding;
* the forces are the exact gradient of the SPME energy (central finite differences);
* E = 1/2 sum q_i phi_i; a shift of every particle by one mesh spacing changes nothing.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import spme
from paper_1708_01135_gb300 import workloads as W


@pytest.mark.parametrize("p", [2, 3, 4, 6, 8])
def test_bspline_partition_symmetry_integral(p):
    u = np.linspace(0.0, 1.0, 37)
    tot = sum(spme.bspline(p, u + k) for k in range(p))
    assert np.abs(tot - 1.0).max() < 1e-14
    if p > 2:
        dtot = sum(spme.bspline_deriv(p, u + k) for k in range(p))
        assert np.abs(dtot).max() < 1e-13
    v = np.linspace(0.0, p, 2001)
    assert np.abs(spme.bspline(p, v) - spme.bspline(p, p - v)).max() < 1e-14
    # trapezoid rule on a fine grid: the splines are smooth enough for 1e-6
    f = spme.bspline(p, v)
    integ = float(((f[1:] + f[:-1]) * 0.5 * np.diff(v)).sum())
    assert abs(integ - 1.0) < 1e-6
    if p == 2:
        assert np.allclose(spme.bspline(2, v), np.maximum(0.0, 1.0 - np.abs(v - 1.0)))


def _system():
    pos, q, L = W.random_neutral(60, density=1.0, hard_core=0.7, seed=3,
                                 mix=((1.0, 0.3), (2.0, 0.2)))
    return pos, q, L


def test_converges_to_classical_ewald():
    pos, q, L = _system()
    beta = 1.2
    kmax = int(math.ceil(6.5 * beta * L / math.pi))
    ek, Fk, pk, _, _ = oracle.recip(pos, q, L, beta, kmax)
    Wk = oracle.virial_recip(pos, q, L, beta, kmax)
    errs = []
    for K, p in [(8, 4), (16, 4), (16, 6), (24, 8), (32, 10), (48, 12)]:
        r = spme.recip(pos, q, L, beta, K, p)
        errs.append(max(abs(r["E"] - ek) / abs(ek),
                        math.sqrt(((r["F"] - Fk) ** 2).sum() / (Fk ** 2).sum()),
                        np.abs(r["phi"] - pk).max() / np.abs(pk).max(),
                        np.abs(r["W"] - Wk).max() / np.abs(Wk).max()))
    # every refinement gains at least a factor 10, and the finest is at rounding level
    for a, b in zip(errs, errs[1:]):
        assert b < 0.1 * a, errs
    assert errs[-1] < 1e-13, errs


def test_forces_are_minus_gradient_of_spme_energy():
    pos, q, L = _system()
    beta, K, p = 1.2, 12, 6            # a coarse mesh: far from the classical sum
    r = spme.recip(pos, q, L, beta, K, p)
    h = 1e-6
    rng = np.random.default_rng(7)
    for i in rng.choice(len(q), 5, replace=False):
        for a in range(3):
            pp = pos.copy(); pp[i, a] += h
            pm = pos.copy(); pm[i, a] -= h
            fd = -(spme.recip(pp, q, L, beta, K, p)["E"] - spme.recip(pm, q, L, beta, K, p)["E"]) / (2 * h)
            assert abs(fd - r["F"][i, a]) < 1e-6 * np.abs(r["F"]).max()


def test_potential_energy_identity_and_mesh_shift():
    pos, q, L = _system()
    beta, K, p = 1.0, 16, 4
    r = spme.recip(pos, q, L, beta, K, p)
    assert abs(0.5 * float((q * r["phi"]).sum()) - r["E"]) < 1e-12 * abs(r["E"])
    s = spme.recip(pos + np.array([L / K, 0.0, 2 * L / K]), q, L, beta, K, p)
    assert abs(s["E"] - r["E"]) < 1e-12 * abs(r["E"])
    assert np.abs(s["F"] - r["F"]).max() < 1e-11 * np.abs(r["F"]).max()
    # an odd order is refused (its Euler spline vanishes at m = K/2)
    with pytest.raises(ValueError):
        spme.recip(pos, q, L, beta, K, 5)


def test_subset_and_blocked_mesh_match_the_whole():
    """Forces of a particle subset equal those rows of the full evaluation, and the charge
    mesh does not depend on how many particles are added per block (one point at a time per
    particle, in particle order, either way)."""
    pos, q, L = W.random_neutral(300, density=1.0, hard_core=0.8, seed=41)
    full = spme.recip(pos, q, L, 1.1, 20, 6)
    sub = np.array([7, 3, 250, 0])
    part = spme.recip(pos, q, L, 1.1, 20, 6, sub=sub)
    assert np.array_equal(part["F"], full["F"][sub])
    assert np.array_equal(part["phi"], full["phi"][sub])
    assert part["E"] == full["E"]
    assert np.array_equal(spme.charge_mesh(pos, q, L, 20, 6, block=1), full["Q"])
