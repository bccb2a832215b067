"""Pins of the oracle's Lennard-Jones pairs (ewo_lj) against facts that fix the pair
potential and its sums, none of which restates the oracle's formulas:

* lattice sums: with two pair sizes sigma the energy separates into its (sigma/d)^12 and
  (sigma/d)^6 parts; the former, per particle, is half the simple-cubic and face-centred-cubic
  lattice sums of Lennard-Jones and Ingham (tests/golden/lj_lattice_sums.txt) for a
  rock-salt grid with one type, and with unlike pairs switched off (each ion species alone
  is an fcc lattice of nearest-neighbour distance sqrt 2);
* the pair potential: zero force at d = 2^(1/6) sigma, energy difference -eps between
  d = 2^(1/6) sigma and d = sigma, energy -> 0 as d -> r_c (the shift), no pair beyond r_c;
* forces: central differences of the energy;
* virial: central differences of the energy under strain of an isolated cluster (every
  component) and under a uniform scaling of a periodic system (the trace);
* types: relabelling the types together with the tables changes nothing.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1708_01135_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sums():
    rows = {}
    with open(os.path.join(GOLDEN, "lj_lattice_sums.txt")) as f:
        for line in f:
            p = line.split("#")[0].split()
            if p:
                rows[p[0]] = (float(p[1]), float(p[2]))
    return rows


def _split_12_6(pos, types, eps, L, rc, s1=0.8, s2=0.9):
    """Coefficients (C12, C6) of E(sigma) / (4 eps) = sigma^12 C12 - sigma^6 C6, from the energies
    at two sizes (every pair gets the same sigma)."""
    T = eps.shape[0]
    e1, _, _ = O.lj(pos, types, eps, np.full((T, T), s1), L, rc)
    e2, _, _ = O.lj(pos, types, eps, np.full((T, T), s2), L, rc)
    A = np.array([[s1 ** 12, -s1 ** 6], [s2 ** 12, -s2 ** 6]])
    return np.linalg.solve(A, np.array([e1, e2]) / 4.0)


def test_simple_cubic_lattice_sum():
    pos, q, L = W.rocksalt(10)                       # a simple cubic grid of spacing 1
    c12, _ = _split_12_6(pos, np.zeros(len(q), dtype=np.int32), np.ones((1, 1)), L, 4.0)
    a12, _ = _sums()["sc"]
    assert abs(c12 / len(q) - a12 / 2) < 2e-5 * a12


def test_fcc_sublattices_when_unlike_pairs_are_off():
    pos, q, L = W.rocksalt(10)
    types = (q < 0).astype(np.int32)
    eps = np.array([[1.0, 0.0], [0.0, 1.0]])
    c12, _ = _split_12_6(pos, types, eps, L, 4.5)
    a12, _ = _sums()["fcc"]
    # each species: fcc with nearest-neighbour distance sqrt(2)
    assert abs(c12 / len(q) - a12 / 2 / np.sqrt(2.0) ** 12) < 2e-5 * a12 / 64


def test_pair_minimum_zero_and_cutoff():
    L, rc, sig, ep = 20.0, 5.0, 1.1, 0.7
    tab_e, tab_s = np.array([[ep]]), np.array([[sig]])

    def pair(d):
        pos = np.array([[5.0, 5.0, 5.0], [5.0 + d / np.sqrt(2), 5.0 + d / np.sqrt(2), 5.0]])
        return O.lj(pos, np.zeros(2, dtype=np.int32), tab_e, tab_s, L, rc)

    rmin = 2 ** (1 / 6) * sig
    e_min, F_min, _ = pair(rmin)
    e_sig, F_sig, _ = pair(sig)
    assert np.abs(F_min).max() < 1e-12
    assert abs((e_min - e_sig) - (-ep)) < 1e-12
    assert F_sig[0, 0] < 0 and F_sig[1, 0] > 0       # repulsive inside the minimum
    assert abs(pair(rc * (1 - 1e-9))[0]) < 1e-9      # the shifted potential vanishes at r_c
    e_out, F_out, W_out = pair(rc * (1 + 1e-9))
    assert e_out == 0.0 and np.all(F_out == 0.0) and np.all(W_out == 0.0)


def _fluid(seed=41):
    pos, q, L = W.random_neutral(300, density=0.9, hard_core=0.85, seed=seed)
    types = (q < 0).astype(np.int32)
    eps = np.array([[0.3, 0.5], [0.5, 0.2]])
    sigma = np.array([[0.9, 0.8], [0.8, 1.0]])
    return pos, types, eps, sigma, L


def test_forces_are_minus_energy_gradient():
    pos, types, eps, sigma, L = _fluid()
    rc = 0.45 * L
    e, F, _ = O.lj(pos, types, eps, sigma, L, rc)
    h = 1e-6
    rng = np.random.default_rng(42)
    for i in rng.choice(len(types), 6, replace=False):
        for a in range(3):
            pp = pos.copy(); pp[i, a] += h
            pm = pos.copy(); pm[i, a] -= h
            fd = -(O.lj(pp, types, eps, sigma, L, rc)[0] - O.lj(pm, types, eps, sigma, L, rc)[0]) / (2 * h)
            assert abs(fd - F[i, a]) < 1e-6 * np.abs(F).max()
    assert np.abs(F.sum(axis=0)).max() < 1e-10 * np.abs(F).max()


def test_virial_matches_strain_derivatives():
    # every component: an isolated cluster (diameter < r_c, no image inside r_c)
    frag, q, _ = W.rocksalt(4, 1.05, 0.08, seed=43)
    types = (q < 0).astype(np.int32)
    eps = np.array([[0.3, 0.5], [0.5, 0.2]])
    sigma = np.array([[0.9, 0.8], [0.8, 1.0]])
    c0 = np.array([12.0, 12.0, 12.0])
    pos = frag - frag.mean(axis=0) + c0
    L, rc = 24.0, 7.0
    _, _, Wt = O.lj(pos, types, eps, sigma, L, rc)
    h = 1e-6
    for a in range(3):
        for b in range(a, 3):
            E = np.zeros((3, 3)); E[a, b] = E[b, a] = 1.0
            ep = O.lj(c0 + (pos - c0) @ (np.eye(3) + h * E).T, types, eps, sigma, L, rc)[0]
            em = O.lj(c0 + (pos - c0) @ (np.eye(3) - h * E).T, types, eps, sigma, L, rc)[0]
            assert abs((E * Wt).sum() + (ep - em) / (2 * h)) < 1e-6 * np.abs(Wt).max()
    # the trace in a periodic fluid: scale coordinates and box together
    pos, types, eps, sigma, L = _fluid(44)
    rc = 0.45 * L
    _, _, Wt = O.lj(pos, types, eps, sigma, L, rc)
    h = 1e-7
    ep = O.lj(pos * (1 + h), types, eps, sigma, L * (1 + h), rc)[0]
    em = O.lj(pos * (1 - h), types, eps, sigma, L * (1 - h), rc)[0]
    assert abs(np.trace(Wt) + (ep - em) / (2 * h)) < 1e-5 * np.abs(Wt).max()


def test_type_relabelling_is_invariant():
    pos, types, eps, sigma, L = _fluid(45)
    rc = 0.4 * L
    a = O.lj(pos, types, eps, sigma, L, rc)
    perm = np.array([1, 0])
    b = O.lj(pos, 1 - types, eps[np.ix_(perm, perm)], sigma[np.ix_(perm, perm)], L, rc)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    with pytest.raises(ValueError):
        O.lj(pos, types + 5, eps, sigma, L, rc)
