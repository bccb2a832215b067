"""Smooth particle-mesh Ewald (ewald_set_spme) against the SPME oracle (oracle/spme.py) on
the FP64, mixed and FP32 plans: reciprocal energy, forces, potentials and virial at several
mesh sizes (powers of two, even and odd non-powers) and orders; the whole evaluation
against the classical oracle at a fine mesh; bit-identical repeats; switching back to the
classical sum; MD with SPME forces."""
import math

import numpy as np
import pytest

from gpu_common import dev, need_gpu, rel, rel_rms, assert_close, torch

import oracle
from oracle import spme as ospme
from paper_1708_01135_gb300 import MD_RECORD, PART_ALL, PART_RECIP, Ewald, EwaldError
from paper_1708_01135_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "mixed": 1e-5, "fp32": 1e-5}


def _eval(ew, pos, q, parts=PART_ALL):
    n = len(q)
    P, Q = dev(pos), dev(q)
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    V = torch.empty((4, 3, 3), dtype=torch.float64, device="cuda")
    E = torch.empty(4, dtype=torch.float64, device="cuda")
    ew.compute_phi_async(P, Q, F, phi, E, parts=parts)
    assert ew.status() == 0
    E1 = torch.empty(4, dtype=torch.float64, device="cuda")
    F1 = torch.empty_like(F)
    ew.compute_virial_async(P, Q, F1, V, E1, parts=parts)
    assert ew.status() == 0
    return F.cpu().numpy(), phi.cpu().numpy(), V.cpu().numpy(), E.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("K,order", [(32, 6), (30, 4), (45, 8), (24, 12)])
def test_spme_recip_matches_oracle(precision, K, order):
    need_gpu()
    pos, q, L = W.random_neutral(2000, density=1.0, hard_core=0.8, seed=61,
                                 mix=((1.0, 0.4), (2.0, 0.1)))
    beta, rc = 0.8, 0.3 * L
    ref = ospme.recip(pos, q, L, beta, K, order)
    with Ewald(L, beta, rc, 8, precision) as ew:
        ew.set_spme(K, order)
        F, phi, V, E = _eval(ew, pos, q, PART_RECIP)
    tol = TOL[precision]
    assert rel(E[1], ref["E"]) < tol
    assert_close(F, ref["F"], tol)
    assert_close(phi, ref["phi"], tol)
    assert np.abs(V[1] - ref["W"]).max() < tol * np.abs(ref["W"]).max()
    assert E[0] == 0.0 and E[2] == 0.0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spme_total_approaches_classical_ewald(precision):
    """At a fine mesh (K = 64, p = 10 on a box of 12.6) SPME reproduces the classical sum."""
    need_gpu()
    pos, q, L = W.random_neutral(2000, density=1.0, hard_core=0.8, seed=62)
    beta, rc = 0.9, 0.4 * L
    kmax = int(math.ceil(6.5 * beta * L / math.pi))
    ref = oracle.ewald(pos, q, L, beta, rc, kmax)
    with Ewald(L, beta, rc, kmax, precision) as ew:
        ew.set_spme(64, 10)
        F, phi, V, E = _eval(ew, pos, q)
    tol = 1e-8 if precision == "fp64" else 1e-5
    assert_close(F, ref["F"], tol)
    assert rel(E[3], ref["E_total"]) < tol


def test_spme_repeatable_switch_back_and_md():
    need_gpu()
    pos, q, L = W.random_neutral(4000, density=1.0, hard_core=0.8, seed=63)
    beta, rc, kmax = 0.85, 0.25 * L, 14
    with Ewald(L, beta, rc, kmax, "mixed") as plain:
        F0, phi0, V0, E0 = _eval(plain, pos, q)
    with Ewald(L, beta, rc, kmax, "mixed") as ew:
        ew.set_spme(32, 6)
        a = _eval(ew, pos, q)
        b = _eval(ew, pos, q)
        with pytest.raises(EwaldError):
            ew.structure_factor()
        ew.set_spme(0)
        c = _eval(ew, pos, q)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    for x, y in zip(c, (F0, phi0, V0, E0)):
        assert np.array_equal(x, y)
    assert_close(a[0], F0, 1e-2)         # SPME at K = 32, p = 6 is close to the k-space sum


def _md_drift(ew, pos, q, steps=200, dt=1e-3):
    tp, tv = dev(pos), torch.zeros((len(q), 3), dtype=torch.float64, device="cuda")
    Fm = torch.empty_like(tp)
    log = torch.empty((steps + 1, MD_RECORD), dtype=torch.float64, device="cuda")
    ew.md(tp, tv, dev(q), Fm, dt, steps, log=log)
    assert ew.status() == 0
    lg = log.cpu().numpy()
    return np.abs(lg[:, 5] - lg[0, 5]).max() / abs(lg[0, 3]), lg[-1, 4]


def test_spme_md_conserves_energy():
    """Jittered rock-salt 16^3 from rest, 200 steps of dt = 1e-3 on SPME forces (K = 32,
    p = 6): the energy is conserved as well as with the classical k-space sum."""
    need_gpu()
    pos, q, L = W.rocksalt(16, 1.0, 0.05, seed=77)
    with Ewald(L, 0.75, 5.0, 14, "mixed") as ew:
        d_classic, _ = _md_drift(ew, pos, q)
        ew.set_spme(32, 6)
        d_spme, ke = _md_drift(ew, pos, q)
    print(f"MD drift over 200 steps: classical {d_classic:.2e}, SPME {d_spme:.2e}")
    assert ke > 0 and d_spme < 1e-7 and d_classic < 1e-7


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spme_single_cell_grid_spreads_particle_by_particle(precision):
    """r_c = L/2 on a small box leaves the real-space grid a single cell (all pairs), too
    coarse for brick tiles, so the charges are spread particle by particle; the result is the
    same SPME sum (oracle) as with tiles."""
    need_gpu()
    pos, q, L = W.random_neutral(500, density=1.0, hard_core=0.8, seed=64)
    beta, rc = 0.9, 0.5 * L
    ref = ospme.recip(pos, q, L, beta, 24, 6)
    with Ewald(L, beta, rc, 8, precision) as ew:
        ew.set_spme(24, 6)
        F, phi, V, E = _eval(ew, pos, q, PART_RECIP)
    tol = TOL[precision]
    assert rel(E[1], ref["E"]) < tol
    assert_close(F, ref["F"], tol)
    assert_close(phi, ref["phi"], tol)
