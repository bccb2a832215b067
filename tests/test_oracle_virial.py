"""Pins of the oracle's virial tensors (W_ab = -dE/d(eps_ab) at fixed beta) against facts
that the mathematics fixes, none of which restates the oracle's formulas:

* trace: scaling every coordinate and the box by lambda multiplies each separation and each
  k by lambda and 1/lambda; -dE/dlambda at lambda = 1, taken by central differences of the
  oracle's energies, is tr W of the real and of the reciprocal part separately (periodic
  systems, with the all-images loop and with the minimum image);
* every component of the real-space tensor: an isolated cluster in a large box (no image
  within the cutoff) strained by (1 + h E) gives -dE_real/dh = sum_ab E_ab W_ab;
* the Coulomb virial identity: the point-charge energy is homogeneous of degree -1, so at
  converged cutoffs tr(W_real + W_recip) = E_real + E_recip + E_self;
* beta invariance: W_real + W_recip does not depend on beta at converged cutoffs, component
  by component, although each part does (this pins the anisotropic reciprocal terms);
* cubic symmetry: the perfect rock-salt lattice has W = (E/3) I with E fixed by its
  Madelung constant (tests/golden/madelung.txt).
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1708_01135_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _madelung(name):
    with open(os.path.join(GOLDEN, "madelung.txt")) as f:
        for line in f:
            parts = line.split("#")[0].split()
            if parts and parts[0] == name:
                return [float(x) for x in parts[1:]]
    raise KeyError(name)


def _converged(L, beta, p=6.5):
    return p / beta, int(math.ceil(p * beta * L / math.pi))


def _systems():
    # rock-salt 4^3 (all-images loop: r_c > L/2), 40 random ions (all-images loop), and 400
    # random ions with r_c <= L/2 (minimum image)
    a = W.rocksalt(4, 1.0, 0.07, seed=21) + (1.3,)
    b = W.random_neutral(40, density=1.0, hard_core=0.7, mix=((1.0, 0.3), (2.0, 0.2)), seed=22) + (1.2,)
    c = W.random_neutral(400, density=1.0, hard_core=0.7, seed=23) + (1.9,)
    return [a, b, c]


def _energies(pos, q, L, beta, rc, kmax):
    er, _, _ = O.real(pos, q, L, beta, rc)
    ek, _, _, _, _ = O.recip(pos, q, L, beta, kmax)
    return er, ek


@pytest.mark.parametrize("which", [0, 1, 2])
def test_virial_trace_is_minus_scaling_derivative(which):
    pos, q, L, beta = _systems()[which]
    rc, kmax = _converged(L, beta)
    if which == 2:
        assert rc <= L / 2      # the minimum-image branch
    else:
        assert rc > L / 2       # the all-images branch
    Wr = O.virial_real(pos, q, L, beta, rc)
    Wk = O.virial_recip(pos, q, L, beta, kmax)
    h = 1e-5
    erp, ekp = _energies(pos * (1 + h), q, L * (1 + h), beta, rc, kmax)
    erm, ekm = _energies(pos * (1 - h), q, L * (1 - h), beta, rc, kmax)
    dr = -(erp - erm) / (2 * h)
    dk = -(ekp - ekm) / (2 * h)
    scale = abs(erp) + abs(ekp)
    assert abs(np.trace(Wr) - dr) < 1e-8 * scale
    assert abs(np.trace(Wk) - dk) < 1e-8 * scale
    # the parts are not trivially small
    assert abs(np.trace(Wr)) > 1e-3 * scale and abs(np.trace(Wk)) > 1e-3 * scale


def test_real_virial_components_match_cluster_strain():
    # a jittered 4^3 rock-salt fragment (diameter ~6.4) in a box of 30 with r_c = 8: every pair
    # of the cluster is inside the cutoff and no image is
    frag, q, _ = W.rocksalt(4, 1.2, 0.1, seed=24)
    c0 = np.array([15.0, 14.0, 16.0])
    pos = frag - frag.mean(axis=0) + c0
    L, beta, rc = 30.0, 0.45, 8.0
    d = np.linalg.norm(pos[:, None] - pos[None], axis=2)
    assert d.max() < rc and L - d.max() > rc
    Wr = O.virial_real(pos, q, L, beta, rc)
    h = 1e-5
    for a in range(3):
        for b in range(a, 3):
            E = np.zeros((3, 3))
            E[a, b] = E[b, a] = 1.0
            ep, _, _ = O.real(c0 + (pos - c0) @ (np.eye(3) + h * E).T, q, L, beta, rc)
            em, _, _ = O.real(c0 + (pos - c0) @ (np.eye(3) - h * E).T, q, L, beta, rc)
            want = -(ep - em) / (2 * h)
            got = (E * Wr).sum()
            assert abs(got - want) < 1e-8 * abs(ep), (a, b, got, want)
    # the off-diagonal part of a jittered cluster is not zero
    assert np.abs(Wr - np.diag(np.diag(Wr))).max() > 1e-3


@pytest.mark.parametrize("which", [0, 1])
def test_virial_identity_and_beta_invariance(which):
    pos, q, L, _ = _systems()[which]
    Ws, Wrs = [], []
    for beta in (0.9, 1.4, 2.2):
        rc, kmax = _converged(L, beta)
        Wr = O.virial_real(pos, q, L, beta, rc)
        Wk = O.virial_recip(pos, q, L, beta, kmax)
        r = O.ewald(pos, q, L, beta, rc, kmax)
        Wt = Wr + Wk
        # the Coulomb energy is homogeneous of degree -1 in the coordinates
        assert abs(np.trace(Wt) - r["E_total"]) < 1e-10 * abs(r["E_total"])
        Ws.append(Wt)
        Wrs.append(Wr)
    scale = np.abs(Ws[0]).max()
    for Wt in Ws[1:]:
        assert np.abs(Wt - Ws[0]).max() < 1e-10 * scale
    # each part moves with beta, also off the diagonal
    assert np.abs(Wrs[2] - Wrs[0]).max() > 1e-2 * scale
    off = ~np.eye(3, dtype=bool)
    assert np.abs((Wrs[2] - Wrs[0])[off]).max() > 1e-4 * scale


@pytest.mark.parametrize("beta", [1.0, 1.8])
def test_rocksalt_virial_is_isotropic_madelung(beta):
    M, r0 = _madelung("NaCl")
    pos, q, L = W.rocksalt(4, a=r0)
    rc, kmax = _converged(L, beta)
    Wt = O.virial_real(pos, q, L, beta, rc) + O.virial_recip(pos, q, L, beta, kmax)
    E = -M / (2 * r0) * len(q)
    assert np.abs(Wt - E / 3 * np.eye(3)).max() < 1e-10 * abs(E)
