"""Pins of the FP64 CPU oracle against facts that the paper and the mathematics fix.

None of these tests compares the oracle with itself: each checks it against a printed
constant, an exact lattice result, an invariance of the exact method, a conservation law,
a finite-difference derivative or an independent brute-force lattice sum.  Together they
catch a dropped term, a wrong sign or factor, or a wrong index in every oracle function:

* real-space sum (Section 3.1.1, Eq. 4): Madelung constants, beta invariance, brute-force
  sums, finite differences of E_real, sum of forces;
* structure factor (Section 3.1.2, Algorithm 1): the exact S(k) of an unjittered
  rock-salt lattice, and the same lattice with positions shifted by whole lattice vectors;
* reciprocal energy and forces (Eq. 3, Algorithm 2): Madelung, beta invariance, finite
  differences of E_recip, sum of forces, the potential/energy identity;
* self energy (Section 3.2.2): beta invariance of the total (it is the only term that
  compensates the beta dependence of the k-space self-interaction);
* k-set: lattice-point counts (tests/golden/lattice_points.txt) and the half-space property.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1708_01135_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_table(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                parts = line.split()
                rows[parts[0]] = [float(x) for x in parts[1:]]
    return rows


def _converged(L, beta, p=6.5):
    """Cutoffs at which both truncation errors are below double rounding: erfc(beta rc) and
    exp(-(pi kmax / (beta L))^2) both below ~1e-18 for p = 6.5."""
    rc = p / beta
    kmax = int(math.ceil(p * beta * L / math.pi))
    return rc, kmax


def _rel_rms(a, b):
    return math.sqrt(float(((a - b) ** 2).sum()) / float((b ** 2).sum()))


# ---- k-set ---------------------------------------------------------------------------

def test_kset_counts_match_lattice_point_table():
    table = _golden_table("lattice_points.txt")
    for r, (count,) in table.items():
        r = int(r)
        if r == 0:
            continue
        assert len(O.kset_half(r)) == (int(count) - 1) // 2


def test_kset_is_a_half_space():
    kmax = 7
    m = O.kset_half(kmax)
    s = {tuple(v) for v in m.tolist()}
    assert len(s) == len(m)
    a = np.arange(-kmax, kmax + 1)
    full = {(x, y, z) for x in a for y in a for z in a if 0 < x * x + y * y + z * z <= kmax * kmax}
    neg = {(-x, -y, -z) for (x, y, z) in s}
    assert s.isdisjoint(neg)
    assert s | neg == full


# ---- Madelung constants --------------------------------------------------------------

@pytest.mark.parametrize("m", [2, 4, 6])
@pytest.mark.parametrize("beta", [1.0, 1.7])
def test_rocksalt_madelung(m, beta):
    M, r0 = _golden_table("madelung.txt")["NaCl"]
    pos, q, L = W.rocksalt(m, a=r0)
    rc, kmax = _converged(L, beta)
    r = O.ewald(pos, q, L, beta, rc, kmax)
    e_per_ion = r["E_total"] / len(q)
    assert abs(e_per_ion - (-M / (2 * r0))) < 1e-12
    # every ion of the perfect lattice is a centre of inversion symmetry: no net force
    assert np.abs(r["F"]).max() < 1e-11


@pytest.mark.parametrize("beta", [1.2, 2.0])
def test_cscl_madelung(beta):
    M, r0c = _golden_table("madelung.txt")["CsCl"]
    c = 1.3
    pos, q, L = W.cscl(3, c=c)
    rc, kmax = _converged(L, beta)
    r = O.ewald(pos, q, L, beta, rc, kmax)
    r0 = r0c * c
    assert abs(r["E_total"] / len(q) - (-M / (2 * r0))) < 1e-11


# ---- exact structure factor of the unjittered lattice --------------------------------

def test_rocksalt_structure_factor_is_exact():
    m = 8
    pos, q, L = W.rocksalt(m)
    km = O.kset_half(8)
    S = O.structure_factor(pos, q, L, km)
    # S(n) = prod_a sum_i (-1)^i e^{2 pi i n_a i / m} = N when every n_a = m/2 (mod m), else 0
    hit = np.all((km % m) == m // 2, axis=1)
    assert hit.sum() == 4  # (+-4, +-4, 4) in the half space
    assert np.allclose(S[hit], len(q), atol=1e-9)
    assert np.abs(S[~hit]).max() < 1e-9
    # shifting every ion by a whole box vector does not change S (periodic phases)
    S2 = O.structure_factor(pos + L * np.array([1.0, -2.0, 3.0]), q, L, km)
    assert np.abs(S2 - S).max() < 1e-9


def test_structure_factor_of_a_single_charge():
    # one charge: S(k) = q exp(i k.r), |S| = |q| for every k; and the phase advances as
    # the position moves by one lattice vector component times the mode number
    L = 3.0
    km = O.kset_half(3)
    r = np.array([[0.4, 1.1, 2.9]])
    S = O.structure_factor(r, np.array([2.0]), L, km)
    assert np.allclose(np.abs(S), 2.0, atol=1e-13)
    S_shift = O.structure_factor(r + np.array([[0.3, 0.0, 0.0]]), np.array([2.0]), L, km)
    expected = S * np.exp(1j * 2 * np.pi * km[:, 0] * 0.3 / L)
    assert np.abs(S_shift - expected).max() < 1e-12


# ---- beta invariance, conservation, derivatives --------------------------------------

def _small_systems():
    pos1, q1, L1 = W.rocksalt(4, 1.0, 0.07, seed=11)
    pos2, q2, L2 = W.random_neutral(40, density=1.0, hard_core=0.7, mix=((1.0, 0.3), (2.0, 0.2)),
                                    seed=12)
    return [(pos1, q1, L1), (pos2, q2, L2)]


@pytest.mark.parametrize("which", [0, 1])
def test_total_is_independent_of_beta(which):
    pos, q, L = _small_systems()[which]
    Es, Fs = [], []
    for beta in (0.9, 1.4, 2.2):
        rc, kmax = _converged(L, beta)
        r = O.ewald(pos, q, L, beta, rc, kmax)
        Es.append(r["E_total"])
        Fs.append(r["F"])
        # the components do depend on beta: the invariance is not trivial
    assert max(Es) - min(Es) < 1e-10 * abs(Es[0])
    for F in Fs[1:]:
        assert _rel_rms(F, Fs[0]) < 1e-10


def test_components_change_with_beta():
    pos, q, L = _small_systems()[0]
    a = O.ewald(pos, q, L, 1.0, *_converged(L, 1.0))
    b = O.ewald(pos, q, L, 2.0, *_converged(L, 2.0))
    for key in ("E_real", "E_recip", "E_self"):
        assert abs(a[key] - b[key]) > 1e-3


@pytest.mark.parametrize("which", [0, 1])
def test_forces_sum_to_zero(which):
    pos, q, L = _small_systems()[which]
    r = O.ewald(pos, q, L, 1.1, 3.5, 9)  # truncated cutoffs: each part still conserves momentum
    for key in ("F_real", "F_recip"):
        F = r[key]
        assert np.abs(F.sum(axis=0)).max() < 1e-12 * len(q) * np.abs(F).max()


def _energy_parts(pos, q, L, beta, rc, kmax):
    r = O.ewald(pos, q, L, beta, rc, kmax)
    return r["E_real"], r["E_recip"]


@pytest.mark.parametrize("which", [0, 1])
def test_forces_are_minus_energy_gradient(which):
    pos, q, L = _small_systems()[which]
    beta = 1.3
    rc, kmax = _converged(L, beta)
    r = O.ewald(pos, q, L, beta, rc, kmax)
    h = 1e-5
    rng = np.random.default_rng(3 + which)
    for i in rng.choice(len(q), 5, replace=False):
        for a in range(3):
            pp = pos.copy(); pp[i, a] += h
            pm = pos.copy(); pm[i, a] -= h
            er_p, ek_p = _energy_parts(pp, q, L, beta, rc, kmax)
            er_m, ek_m = _energy_parts(pm, q, L, beta, rc, kmax)
            fr = -(er_p - er_m) / (2 * h)
            fk = -(ek_p - ek_m) / (2 * h)
            scale = np.abs(r["F"]).max()
            assert abs(fr - r["F_real"][i, a]) < 1e-6 * scale
            assert abs(fk - r["F_recip"][i, a]) < 1e-6 * scale


def test_recip_potential_matches_energy():
    pos, q, L = _small_systems()[1]
    r = O.ewald(pos, q, L, 1.2, 3.0, 8)
    assert abs(0.5 * float((q * r["phi_recip"]).sum()) - r["E_recip"]) < 1e-12 * abs(r["E_recip"])
    assert abs(0.5 * float((q * r["phi_real"]).sum()) - r["E_real"]) < 1e-12 * abs(r["E_real"])


def test_subset_matches_full():
    pos, q, L = _small_systems()[1]
    full = O.ewald(pos, q, L, 1.2, 3.0, 8)
    sub = np.array([3, 17, 0, 39])
    part = O.ewald(pos, q, L, 1.2, 3.0, 8, sub=sub)
    assert np.abs(part["F"] - full["F"][sub]).max() < 1e-13


# ---- brute-force lattice sums ---------------------------------------------------------

def test_cube_sum_of_rocksalt_cell_gives_madelung():
    M, _ = _golden_table("madelung.txt")["NaCl"]
    pos, q, L = W.rocksalt(2)
    E, _ = O.coulomb_cube(pos, q, L, 40)
    assert abs(E[40] / len(q) - (-M / 2)) < 1e-8


def test_cube_sum_matches_ewald_plus_dipole_term():
    rng = np.random.default_rng(5)
    L = 2.0
    pos = rng.uniform(0, L, size=(6, 3))
    q = np.array([1.0, -1.0, 2.0, -2.0, 1.0, -1.0])
    V = L ** 3
    Mdip = (q[:, None] * pos).sum(axis=0)
    beta = 2.0
    r = O.ewald(pos, q, L, beta, *_converged(L, beta))
    E, F = O.coulomb_cube(pos, q, L, 60, forces=True)
    _, F30 = O.coulomb_cube(pos, q, L, 30, forces=True)
    # shells converge as 1/s^2 for a cell with a quadrupole: Richardson on s = 30, 60
    e_inf = (4 * E[60] - E[30]) / 3
    f_inf = (4 * F - F30) / 3
    surface = 2 * math.pi * float(Mdip @ Mdip) / (3 * V)
    assert abs(e_inf - surface - r["E_total"]) < 2e-6 * abs(r["E_total"])
    f_ewald_cube = r["F"] - 4 * math.pi / (3 * V) * q[:, None] * Mdip[None, :]
    assert np.abs(f_inf - f_ewald_cube).max() < 2e-5 * np.abs(r["F"]).max()


def test_pair_in_large_box_approaches_bare_coulomb():
    # a +-1 pair at separation d in a box much larger than d: E -> -1/d plus the periodic
    # correction, which is O(d^2 / L^3); the force -> the bare Coulomb force
    d = 0.7
    L = 40.0
    pos = np.array([[20.0, 20.0, 20.0], [20.0 + d, 20.0, 20.0]])
    q = np.array([1.0, -1.0])
    beta = 0.25
    r = O.ewald(pos, q, L, beta, *_converged(L, beta))
    assert abs(r["E_total"] - (-1.0 / d)) < 1e-3
    assert abs(r["F"][0, 0] - (1.0 / d ** 2)) < 1e-3


@pytest.mark.parametrize("n,L,rc,seed", [(3000, 15.0, 5.0, 3), (2000, 13.7, 4.1, 4), (1200, 11.0, 3.0, 5)])
def test_cell_list_real_space_equals_all_pairs(n, L, rc, seed):
    """The binned real-space sum visits exactly the pairs of the all-pairs loop: the results
    agree to rounding (3 cells per side with L/r_c an integer, ragged cells, 3 cells at
    L/r_c = 3.34, and particles given outside [0, L))."""
    pos, q, L = W.random_neutral(n, L=L, hard_core=0.7, seed=seed, mix=((1.0, 0.4), (2.0, 0.1)))
    pos = pos + L * np.random.default_rng(seed).integers(-2, 3, size=pos.shape)
    e0, F0, p0 = O.real(pos, q, L, 0.9, rc)
    e1, F1, p1 = O.real_cells(pos, q, L, 0.9, rc)
    assert abs(e1 - e0) <= 1e-12 * abs(e0)
    assert np.abs(F1 - F0).max() <= 1e-12 * np.abs(F0).max()
    assert np.abs(p1 - p0).max() <= 1e-12 * np.abs(p0).max()
    sub = np.array([0, 7, n // 2, n - 1])
    _, Fs, ps = O.real_cells(pos, q, L, 0.9, rc, sub=sub)
    assert np.array_equal(Fs, F1[sub]) and np.array_equal(ps, p1[sub])


def test_cell_list_rejects_too_few_cells():
    pos, q, L = W.rocksalt(4)
    with pytest.raises(ValueError):
        O.real_cells(pos, q, L, 1.0, 1.5)       # floor(4 / 1.5) = 2 cells per side
