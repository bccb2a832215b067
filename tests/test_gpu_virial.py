"""Virial tensors (ewald_compute_virial_async) against the oracle's virial_real and
virial_recip on every path (FP64, mixed, FP32), through the cell-list and the all-pairs
real-space kernels; the Coulomb virial identity tr W = E_total and the isotropic rock-salt
tensor on the device; part masks, n = 0 and bitwise repeatability (graph replay)."""
import math

import numpy as np
import pytest

from gpu_common import dev, need_gpu, rel, rel_rms, assert_close, torch

import oracle
from paper_1708_01135_gb300 import PART_ALL, PART_REAL, PART_RECIP, PART_SELF, Ewald
from paper_1708_01135_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 2e-5, "fp32": 2e-5}


def _run(ew, pos, q, parts=PART_ALL):
    n = len(q)
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    V = torch.full((4, 3, 3), float("nan"), dtype=torch.float64, device="cuda")
    E = torch.empty(4, dtype=torch.float64, device="cuda")
    ew.compute_virial_async(dev(pos), dev(q), F, V, E, parts=parts)
    assert ew.status() == 0
    return F.cpu().numpy(), V.cpu().numpy(), E.cpu().numpy()


def _tensor_err(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


CASES = {
    # 20,000 ions, r_c = L/5: cell-list kernel over many tiles with ragged cells
    "cells": dict(n=20000, seed=31, rc_frac=0.2, beta_rc=3.3, kmax=16),
    # 600 ions, r_c = 0.45 L: fewer than 3 cells of side r_c, all-pairs kernel
    "allpairs": dict(n=600, seed=32, rc_frac=0.45, beta_rc=3.3, kmax=10),
}


@pytest.mark.parametrize("precision", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("case", ["cells", "allpairs"])
def test_virial_matches_oracle(precision, case):
    need_gpu()
    c = CASES[case]
    pos, q, L = W.random_neutral(c["n"], density=1.0, hard_core=0.8, seed=c["seed"],
                                 mix=((1.0, 0.4), (2.0, 0.1)))
    rc = c["rc_frac"] * L
    beta = c["beta_rc"] / rc
    Wr_ref = oracle.virial_real(pos, q, L, beta, rc)
    Wk_ref = oracle.virial_recip(pos, q, L, beta, c["kmax"])
    ref = oracle.ewald(pos, q, L, beta, rc, c["kmax"]) if c["n"] <= 5000 else None
    with Ewald(L, beta, rc, c["kmax"], precision) as ew:
        F, V, E = _run(ew, pos, q)
        F0 = torch.empty((len(q), 3), dtype=torch.float64, device="cuda")
        E0 = torch.empty(4, dtype=torch.float64, device="cuda")
        ew.compute_async(dev(pos), dev(q), F0, E0)
        assert ew.status() == 0
    tol = TOL[precision]
    assert _tensor_err(V[0], Wr_ref) < tol, (V[0], Wr_ref)
    assert _tensor_err(V[1], Wk_ref) < tol, (V[1], Wk_ref)
    assert np.all(V[2] == 0.0)
    assert np.array_equal(V[3], V[0] + V[1])
    for t in V:
        assert np.array_equal(t, t.T)
    # the forces and energies of the virial call are those of the plain call
    assert_close(F, F0.cpu().numpy(), (1e-14 if precision == "fp64" else 1e-6))
    assert np.abs(E - E0.cpu().numpy()).max() <= 1e-9 * np.abs(E).max()
    if ref is not None:
        assert rel(E[3], ref["E_total"]) < tol


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_virial_identity_on_device(precision):
    """At converged cutoffs tr(W_real + W_recip) = E_real + E_recip + E_self."""
    need_gpu()
    pos, q, L = W.rocksalt(12, 1.0, 0.08, seed=33)
    beta = 1.0
    rc, km = 5.5, 21
    with Ewald(L, beta, rc, km, precision) as ew:
        _, V, E = _run(ew, pos, q)
    tol = 1e-9 if precision == "fp64" else TOL[precision]
    assert rel(np.trace(V[3]), E[3]) < tol
    # the two parts are separately far from that identity
    assert rel(np.trace(V[0]), E[0] + E[2]) > 1e-2


def test_rocksalt_virial_is_isotropic():
    need_gpu()
    pos, q, L = W.rocksalt(8)
    with Ewald(L, 1.0, 4.0, 10, "fp64") as ew:
        _, V, E = _run(ew, pos, q)
    M = 1.747564594633182
    want = -M / 2.0 * len(q) / 3.0
    assert np.abs(V[3] - want * np.eye(3)).max() < 1e-6 * abs(want)


def test_virial_parts_empty_and_repeatable():
    need_gpu()
    pos, q, L = W.random_neutral(3002, density=1.0, hard_core=0.8, seed=34)
    rc = 0.25 * L
    with Ewald(L, 3.2 / rc, rc, 12, "mixed") as ew:
        # the same buffers three times: run directly, then captured and replayed as a graph
        P, Q = dev(pos), dev(q)
        F = torch.empty((len(q), 3), dtype=torch.float64, device="cuda")
        V = torch.empty((4, 3, 3), dtype=torch.float64, device="cuda")
        E = torch.empty(4, dtype=torch.float64, device="cuda")
        outs = []
        for _ in range(3):
            V.fill_(float("nan"))
            ew.compute_virial_async(P, Q, F, V, E)
            assert ew.status() == 0
            outs.append(V.cpu().numpy())
        Va, Vb, Vc = outs
        _, Vr, _ = _run(ew, pos, q, PART_REAL)
        _, Vk, _ = _run(ew, pos, q, PART_RECIP)
        _, Vs, _ = _run(ew, pos, q, PART_SELF)
        z = torch.full((4, 3, 3), 7.0, dtype=torch.float64, device="cuda")
        e = torch.full((4,), 7.0, dtype=torch.float64, device="cuda")
        f = torch.empty((0, 3), dtype=torch.float64, device="cuda")
        ew.compute_virial_async(f, torch.empty(0, dtype=torch.float64, device="cuda"), f, z, e)
        assert ew.status() == 0
        assert bool((z == 0).all()) and bool((e == 0).all())
    assert np.array_equal(Va, Vb) and np.array_equal(Va, Vc)
    assert np.array_equal(Vr[0], Va[0]) and np.all(Vr[1] == 0) and np.array_equal(Vr[3], Va[0])
    assert np.array_equal(Vk[1], Va[1]) and np.all(Vk[0] == 0) and np.array_equal(Vk[3], Va[1])
    assert np.all(Vs == 0)
